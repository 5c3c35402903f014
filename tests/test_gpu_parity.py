"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L-inf per field = max|gpu - oracle| / max|oracle|):
FP64 mode 1e-12 per step; FP32 mode 1e-5 after one step, 1e-3 relative L2
in H after 1000 steps, mass drift 1e-6.  FP32 runs get inputs rounded to
FP32 on both sides so only the arithmetic differs.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1705_00614_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1705_00614_gb300 import build, swe as S
    build.build()
    S.load()
    return S


def rel(g, o, floor=1e-300):
    den = max(np.abs(o).max(), floor)
    return np.abs(g - o).max() / den


def assert_state_close(gs, os_, tol, what=""):
    for name, g, o in zip(("H", "Qx", "Qy"), gs, os_):
        err = rel(g, o, floor=1e-6)
        assert err <= tol, f"{what} {name}: rel Linf {err:.3e} > {tol:.1e}"


SHAPES = [(67, 45), (130, 77), (300, 270)]


@pytest.mark.parametrize("nx,ny", SHAPES[:2])
def test_staged_f64_every_stage_matches_oracle(swe, nx, ny):
    """One step of the one-kernel-per-stage mode (the paper's K2-K8 split):
    every intermediate and the new state agree with the oracle's stages."""
    p = I.random_wet_dry(nx, ny, seed=nx + ny)
    Ho, Qxo, Qyo, info, st = oracle.step(p, p.H, p.Qx, p.Qy, 0.0, stages=True)
    with swe.Solver.from_problem(p, "f64", "staged") as s:
        gi = s.step(1)
        gst = s.stages()
        H, Qx, Qy, t = s.get_state()
    assert abs(gi["dt_last"] - info["tau"]) <= 1e-14 * info["tau"]
    for k in swe.STAGE_NAMES:
        err = rel(gst[k], st[k], floor=1e-12)
        assert err <= 1e-12, f"stage {k}: rel Linf {err:.3e}"
    assert_state_close((H, Qx, Qy), (Ho, Qxo, Qyo), 1e-12)
    assert abs(gi["mass"] - info["mass"]) <= 1e-12 * info["mass"]
    assert abs(gi["src_vol"] - info["src_vol"]) <= 1e-9 * max(1.0, abs(info["src_vol"]))


@pytest.mark.parametrize("nx,ny,seg_h", [(67, 45, 0), (130, 77, 8), (300, 270, 16), (233, 129, 24)])
def test_fused_f64_matches_oracle_each_step(swe, nx, ny, seg_h):
    """Fused kernel, FP64, several steps with CFL time steps, sources and
    wet/dry fronts; grids spanning several 116-column strips and row
    segments with ragged tails."""
    p = I.random_wet_dry(nx, ny, seed=3 * nx + ny)
    bd = oracle._Bound(p)
    H, Qx, Qy, t = p.H, p.Qx, p.Qy, 0.0
    with swe.Solver.from_problem(p, "f64", "fused", seg_h=seg_h) as s:
        for n in range(4):
            H, Qx, Qy, info, _ = oracle.step(p, H, Qx, Qy, t, bound=bd)
            t = info["t_new"]
            gi = s.step(1)
            g = s.get_state()
            assert abs(g[3] - t) <= 1e-13 * t
            assert_state_close(g[:3], (H, Qx, Qy), 1e-12, f"step {n}")
            assert abs(gi["mass"] - info["mass"]) <= 1e-12 * info["mass"]
            assert gi["wet_cells"] == info["wet"]


@pytest.mark.parametrize("nx,ny,seg_h", [(130, 77, 0), (300, 270, 16)])
def test_fused_f32_one_step_within_1e5(swe, nx, ny, seg_h):
    p = I.random_wet_dry(nx, ny, seed=7 * nx + ny).to_f32_values()
    Ho, Qxo, Qyo, info, _ = oracle.step(p, p.H, p.Qx, p.Qy, 0.0)
    with swe.Solver.from_problem(p, "f32", "fused", seg_h=seg_h) as s:
        gi = s.step(1)
        g = s.get_state()
    assert abs(gi["dt_last"] - info["tau"]) <= 1e-6 * info["tau"]
    assert_state_close(g[:3], (Ho, Qxo, Qyo), 1e-5)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fused_equals_staged(swe, prec):
    """The fused kernel and the stage-per-kernel mode run the same
    arithmetic: bitwise equal in FP64, within FP32 rounding otherwise."""
    p = I.random_wet_dry(150, 90, seed=11)
    if prec == "f32":
        p = p.to_f32_values()
    with swe.Solver.from_problem(p, prec, "fused", seg_h=16) as a, swe.Solver.from_problem(p, prec, "staged") as b:
        for _ in range(3):
            a.step(1)
            b.step(1)
        ga, gb = a.get_state(), b.get_state()
    if prec == "f64":
        for x, y in zip(ga, gb):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    else:
        assert_state_close(ga[:3], gb[:3], 2e-6)


def test_stoker_dam_break_f64_200_steps(swe):
    """256^2 dam break (h 2 m / 1 m, dx 1 m, K 0.3, 200 steps), GPU FP64:
    every step within 1e-12 of one oracle step from the GPU's own previous
    state; the GPU and oracle trajectories within 1e-12 for the first 20
    steps and 1e-11 after every 20-step block (one-step differences add up);
    exact mass conservation."""
    p = I.dam_break(256, 1.0)
    bd = oracle._Bound(p)
    H, Qx, Qy, t = p.H, p.Qx, p.Qy, 0.0
    g = (H, Qx, Qy, t)
    m0 = 256 * 128 * 3.0
    with swe.Solver.from_problem(p, "f64") as s:
        for n in range(200):
            Hs, Qxs, Qys, info, _ = oracle.step(p, g[0], g[1], g[2], g[3], bound=bd)
            H, Qx, Qy, info_t, _ = oracle.step(p, H, Qx, Qy, t, bound=bd)
            t = info_t["t_new"]
            gi = s.step(1)
            g = s.get_state()
            assert abs(gi["dt_last"] - info["tau"]) <= 1e-14 * info["tau"]
            assert_state_close(g[:3], (Hs, Qxs, Qys), 1e-12, f"step {n + 1} from the GPU state")
            if n < 20 or (n + 1) % 20 == 0:
                assert abs(g[3] - t) <= 1e-12 * t
                assert_state_close(g[:3], (H, Qx, Qy), 1e-12 if n < 20 else 1e-11, f"after {n + 1} steps")
            assert abs(gi["mass"] - m0) <= 1e-13 * m0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_time_step_set_by_particle_speed(swe, prec):
    """Thin uniform flow U = (3, 0) m/s, 1 cm deep, under a -20 m/s wind on
    a flat frictionless bed: the wind stress gives a = -52.9 m/s^2 along x,
    so the particle speed U_p = |U_x - sqrt(h |a_x|)| (11.5 m/s) exceeds the
    wave speed U_s (3.3 m/s) and sets tau = K h / U_p (Fig. 2).  The first
    tau (from the state pass) and the second (from the step's epilogue)
    against the oracle's, and the first against the closed form."""
    n, H0, dx = 40, 0.01, 4.0
    z = np.zeros((n, n))
    par = I.Params(nx=n, ny=n, dx=dx, wind_x=-20.0, wind_y=0.0, c_a=1.0, rho_air_over_rho=1.0e-3,
                   coriolis_f=0.0, nu=0.0, cfl=0.3, dt_max=10.0)
    p = I.Problem("wind", par, z.copy(), z.copy(), np.full((n, n), H0), np.full((n, n), 3.0 * H0),
                  z.copy(), I.Sources.empty())
    ax = 1.0e-3 * (-23.0) * 23.0 / H0
    up = abs(3.0 - math.sqrt(dx * abs(ax)))
    tol = 1e-14 if prec == "f64" else 1e-6
    H, Qx, Qy, t = p.H, p.Qx, p.Qy, 0.0
    with swe.Solver.from_problem(p, prec) as s:
        for k in range(2):
            H, Qx, Qy, info, _ = oracle.step(p, H, Qx, Qy, t)
            t = info["t_new"]
            gi = s.step(1)
            assert abs(gi["dt_last"] - info["tau"]) <= tol * info["tau"], (k, gi["dt_last"], info["tau"])
            if k == 0:
                assert abs(gi["dt_last"] - 0.3 * dx / up) <= tol * (0.3 * dx / up)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_over_draining_sources_match_oracle(swe, prec):
    """Strong drains (rate -60 m/s x weight, against steps of ~0.01 s) that take more water than many
    of their cells hold: those cells keep no momentum (a drain takes water
    with the cell's velocity, never more than the cell holds).  FP64 fused
    and staged per step within 1e-12 of the oracle; FP32 within 1e-5 after
    one step."""
    p = I.random_wet_dry(130, 77, seed=23, drain=-60.0)
    if prec == "f32":
        p = p.to_f32_values()
    _, _, _, info, st = oracle.step(p, p.H, p.Qx, p.Qy, 0.0, stages=True)
    s_ = p.sources
    tau = info["tau"]
    emptied = [(y, x) for x, y, hy, w in zip(s_.ix, s_.iy, s_.hydro, s_.weight)
               if hy == 1 and p.H[y, x] > p.params.eps and p.H[y, x] - 60.0 * w * tau < 0.0
               and abs(st["utx"][y, x]) + abs(st["uty"][y, x]) > 1e-3]
    assert len(emptied) >= 3, "the case must have moving cells emptied by a drain"
    for y, x in emptied:
        assert st["qtx"][y, x] == 0.0 and st["qty"][y, x] == 0.0
    bd = oracle._Bound(p)
    if prec == "f64":
        for mode in ("fused", "staged"):
            H, Qx, Qy, t = p.H, p.Qx, p.Qy, 0.0
            with swe.Solver.from_problem(p, "f64", mode) as s:
                for n in range(4):
                    H, Qx, Qy, info, _ = oracle.step(p, H, Qx, Qy, t, bound=bd)
                    t = info["t_new"]
                    gi = s.step(1)
                    g = s.get_state()
                    assert_state_close(g[:3], (H, Qx, Qy), 1e-12, f"{mode} step {n}")
                    assert abs(gi["src_vol"] - info["src_vol"]) <= 1e-9 * max(1.0, abs(info["src_vol"]))
    else:
        Ho, Qxo, Qyo, info, _ = oracle.step(p, p.H, p.Qx, p.Qy, 0.0, bound=bd)
        with swe.Solver.from_problem(p, "f32", "fused") as s:
            s.step(1)
            g = s.get_state()
        assert_state_close(g[:3], (Ho, Qxo, Qyo), 1e-5)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_lake_at_rest_stays_at_rest(swe, prec):
    p = I.with_gates(I.lake_at_rest(200, 10.0, 7, eta0=12.0), 5, 6)
    with swe.Solver.from_problem(p, prec) as s:
        s.step(200)
        H, Qx, Qy, t = s.get_state()
    assert np.all(Qx == 0.0) and np.all(Qy == 0.0)
    Hr = np.asarray(p.H, dtype=np.float32 if prec == "f32" else np.float64).astype(np.float64)
    assert np.array_equal(H, Hr)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_determinism_graph_and_resume(swe, prec):
    """Same inputs give bitwise-equal results; one 10-step graph equals ten
    single steps; stopping, copying the state out and resuming in a new
    context continues bitwise identically (the speed pass of the new
    context stores the forces the kernel would have stored)."""
    p = I.random_wet_dry(140, 100, seed=17)
    if prec == "f32":
        p = p.to_f32_values()
    with swe.Solver.from_problem(p, prec) as a:
        a.step(10)
        ref = a.get_state()
    with swe.Solver.from_problem(p, prec) as b:
        for _ in range(10):
            b.step(1)
        one = b.get_state()
    with swe.Solver.from_problem(p, prec) as c:
        c.step(4)
        H, Qx, Qy, t = c.get_state()
    with swe.Solver.from_problem(p, prec) as d:
        d.set_state(H, Qx, Qy, t)
        d.step(6)
        res = d.get_state()
    for x, y, z in zip(ref, one, res):
        assert np.array_equal(np.asarray(x), np.asarray(y))
        assert np.array_equal(np.asarray(x), np.asarray(z))


def test_gates_toggle_matches_oracle(swe):
    p = I.with_gates(I.random_wet_dry(120, 96, seed=23), 9, 8)
    p.solid[40:60, 50] = 1
    bd = oracle._Bound(p)
    H, Qx, Qy, t, _ = oracle.run(p, 3)
    with swe.Solver.from_problem(p, "f64") as s:
        s.step(3)
        assert_state_close(s.get_state()[:3], (H, Qx, Qy), 1e-12, "closed")
        # open the wall segment, close two other cells
        iy, ix = np.nonzero(p.solid)
        opened = (ix == 50) & (iy >= 40) & (iy < 60)
        p.solid[40:60, 50] = 0
        p.solid[10, 10:12] = 1
        s.set_solid(np.r_[ix[opened], [10, 11]], np.r_[iy[opened], [10, 10]],
                    np.r_[np.zeros(opened.sum(), np.uint8), [1, 1]].astype(np.uint8))
        H, Qx, Qy, t, _ = oracle.run(p, 3, H, Qx, Qy, t)
        s.step(3)
        assert_state_close(s.get_state()[:3], (H, Qx, Qy), 1e-12, "after toggling")


def test_t_end_lands_exactly_and_stops(swe):
    p = I.dam_break(64, 1.0, ny=8)
    with swe.Solver.from_problem(p, "f64") as s:
        info = s.step(1000, t_end=1.2345)
        assert info["t"] == 1.2345
        n = info["step"]
        info2 = s.step(5, t_end=1.2345)
        assert info2["t"] == 1.2345 and info2["step"] == n
    H, Qx, Qy, t, _ = oracle.run(p, 1000, t_end=1.2345)
    assert t == 1.2345


def test_overflowing_state_is_reported(swe):
    """Depths whose squares overflow FP32 make infinite signal speeds: the
    step reports SWE_ERR_NONFINITE instead of silently continuing."""
    p = I.dam_break(32, 1.0, 3.0e37, 1.0e37, ny=8)
    with swe.Solver.from_problem(p, "f32") as s:
        with pytest.raises(swe.SweError) as e:
            s.step(1)
        assert e.value.code == -4


def test_floodplain_2048_f32_1000_steps(swe):
    """2048^2 floodplain, dx 10 m, fractal terrain with a carved channel,
    Manning patches, viscosity, Coriolis at 48N, wind, a 100-cell Gaussian
    inflow strip, dry start.  The oracle takes 1000 FP64 steps on the window
    that holds all the water (water never comes near the window's edges, so
    walls there change nothing); the GPU runs the full grid in FP32 up to the
    same simulated time (its own CFL steps, landing on it with t_end).  The
    CFL step is set by the fastest signal at thin wet fronts and is itself
    sensitive to FP32 rounding, so states are compared at equal time, not
    equal step count.  Bars: rel L2 of H <= 1e-3; the GPU's FP64 mass budget
    (mass - sources - clipping) drifts by <= 1e-6."""
    full = I.workload("floodplain-2048sq-dx10m").to_f32_values()
    src = full.sources
    j0, j1, i1 = int(src.iy.min()) - 100, int(src.iy.max()) + 100, 200
    crop = I.Problem("crop", I.Params(**{**full.params.__dict__, "nx": i1, "ny": j1 - j0}),
                     full.b[j0:j1, :i1], full.n_manning[j0:j1, :i1], full.H[j0:j1, :i1],
                     full.Qx[j0:j1, :i1], full.Qy[j0:j1, :i1],
                     I.Sources(src.ix, src.iy - j0, src.weight, src.vx, src.vy, src.hydro, src.hydrographs))
    H, Qx, Qy, t, infos = oracle.run(crop, 1000)
    assert np.abs(H[:8]).max() == 0 and np.abs(H[-8:]).max() == 0 and np.abs(H[:, -8:]).max() == 0
    budget = 0.0
    with swe.Solver.from_problem(full, "f32") as s:
        m0 = s.step(0)["mass"]
        steps = 0
        while True:
            gi = s.step(1, t_end=t)
            if gi["step"] == steps:
                break
            steps = gi["step"]
            budget += gi["src_vol"] + gi["clip_vol"]
        Hg, Qxg, Qyg, tg = s.get_state()
    assert tg == t and 950 <= steps <= 1050, (tg, t, steps)
    wet = np.argwhere(Hg > 0.0)
    assert wet[:, 0].min() > j0 + 8 and wet[:, 0].max() < j1 - 8 and wet[:, 1].max() < i1 - 8
    Hc = Hg[j0:j1, :i1]
    l2 = np.linalg.norm(Hc - H) / np.linalg.norm(H)
    assert l2 <= 1e-3, l2
    assert abs(gi["mass"] - (m0 + budget)) <= 1e-6 * gi["mass"]
    assert sum(i["src_vol"] for i in infos) > 0


def test_full_size_16384_sampled_cells(swe):
    """16384^2 floodplain at dx 2 m, flooded to eta = 15 m with seeded
    velocities, one FP32 step (fixed tau) in the benchmark's launch
    configuration.  The new state of sampled cells (random ones and cells on
    the CTA tile and segment seams) is recomputed by the oracle on a
    17x17-cell window around each: one step depends only on cells within 6."""
    n = 16384
    base = I.workload("floodplain-16384sq-dx2m")
    b = base.b
    H = np.maximum(0.0, 15.0 - b).astype(np.float32).astype(np.float64)
    u = I.uniform(77, 1, np.arange(2 * n * n)).reshape(2, n, n)
    Qx = np.where(H > 1e-4, H * (2 * u[0] - 1), 0.0).astype(np.float32).astype(np.float64)
    Qy = np.where(H > 1e-4, H * (2 * u[1] - 1), 0.0).astype(np.float32).astype(np.float64)
    del u
    params = I.Params(**{**base.params.__dict__, "dt_fixed": 0.02})
    prob = I.Problem("flood", params, b.astype(np.float32).astype(np.float64),
                     base.n_manning.astype(np.float32).astype(np.float64), H, Qx, Qy, I.Sources.empty())
    with swe.Solver.from_problem(prob, "f32") as s:
        s.step(1)
        Hg, Qxg, Qyg, t = s.get_state()
    rng = np.random.default_rng(5)
    pts = [(int(y), int(x)) for y, x in rng.integers(0, n, size=(48, 2))]
    pts += [(1000 + d, 116 * k + e) for k, d, e in ((3, 0, -1), (70, 5, 0), (141, 9, 1))]
    pts += [(0, 0), (n - 1, n - 1), (n - 1, 5), (7, n - 1)]
    R = 8
    checked = 0
    for (y, x) in pts:
        y0, y1, x0, x1 = max(0, y - R), min(n, y + R + 1), max(0, x - R), min(n, x + R + 1)
        w = I.Problem("w", I.Params(**{**params.__dict__, "nx": x1 - x0, "ny": y1 - y0}),
                      prob.b[y0:y1, x0:x1], prob.n_manning[y0:y1, x0:x1], H[y0:y1, x0:x1],
                      Qx[y0:y1, x0:x1], Qy[y0:y1, x0:x1], I.Sources.empty())
        Ho, Qxo, Qyo, info, _ = oracle.step(w, w.H, w.Qx, w.Qy, 0.0)
        yy, xx = y - y0, x - x0
        for g, o, sc in ((Hg[y, x], Ho[yy, xx], max(1.0, np.abs(Ho).max())),
                         (Qxg[y, x], Qxo[yy, xx], max(1.0, np.abs(Qxo).max())),
                         (Qyg[y, x], Qyo[yy, xx], max(1.0, np.abs(Qyo).max()))):
            assert abs(g - o) <= 1e-5 * sc, (y, x, g, o)
        checked += 1
    assert checked == len(pts)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_dam_break_rows_identical_and_transposed(swe, prec):
    """A dam break along x over several windows and segments keeps every row
    bitwise equal with zero y momentum; the same dam break along y is its
    transpose (bitwise in FP64; the x and y faces run through different
    code, so FP32 within rounding)."""
    px = I.dam_break(300, 1.0, 2.0, 1.0, ny=70)
    py = I.Problem("dam_break_y", I.Params(**{**px.params.__dict__, "nx": 70, "ny": 300}), px.b.T.copy(),
                   px.n_manning.T.copy(), px.H.T.copy(), px.Qy.T.copy(), px.Qx.T.copy(), I.Sources.empty())
    with swe.Solver.from_problem(px, prec, seg_h=16) as a, swe.Solver.from_problem(py, prec, seg_h=16) as b:
        ia = a.step(60)
        ib = b.step(60)
        Hx, Qxx, Qyx = a.get_state()[:3]
        Hy, Qxy, Qyy = b.get_state()[:3]
    for q in (Hx, Qxx):
        assert np.array_equal(q, np.repeat(q[:1], q.shape[0], axis=0))
    assert not np.asarray(Qyx).any() and not np.asarray(Qxy).any()
    assert ia["t"] == ib["t"]
    if prec == "f64":
        assert np.array_equal(Hy, Hx.T) and np.array_equal(Qyy, Qxx.T)
    else:
        assert_state_close((Hy.T, Qyy.T, Qxy.T), (Hx, Qxx, Qyx), 1e-5)
