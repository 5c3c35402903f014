"""Dry-tile skipping (skip_dry), the wet-block test of the paper's kernel K1
(Sec. 3), through the C ABI.

A work item whose window holds no wet cell and no source is not computed;
the cells it owns keep H and get Q = 0.  Every run below is compared with
the same run without skipping: states and step reports (time, tau, mass,
source and clipped volumes, speed, wet cells) must be bitwise equal, and the
skipping run must really have skipped items.
"""
import dataclasses

import numpy as np
import pytest

from paper_1705_00614_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REPORT_KEYS = ("t", "dt_last", "mass", "src_vol", "clip_vol", "max_speed", "wet_cells", "step", "err_word")


@pytest.fixture(scope="module")
def swe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1705_00614_gb300 import build, swe as S
    build.build()
    S.load()
    return S


def _patchy(nx, ny, seed, prec, centre, radius):
    """Random wet/dry state and all physics on, but water only inside one
    disc: most of the grid is dry."""
    p = I.random_wet_dry(nx, ny, seed=seed, with_sources=False)
    yy, xx = np.mgrid[0:ny, 0:nx]
    inside = (xx - centre[0]) ** 2 + (yy - centre[1]) ** 2 < radius ** 2
    p = dataclasses.replace(p, H=np.where(inside, p.H, 0.0), Qx=np.where(inside, p.Qx, 0.0),
                            Qy=np.where(inside, p.Qy, 0.0))
    return p.to_f32_values() if prec == "f32" else p


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def _same_reports(ra, rb):
    for x, y in zip(ra, rb):
        for k in REPORT_KEYS:
            assert x[k] == y[k], (k, x[k], y[k])


def _run(swe, prob, prec, chunks, skip, seg_h=32, between=None):
    reps = []
    with swe.Solver.from_problem(prob, prec, seg_h=seg_h, skip_dry=skip) as s:
        for i, n in enumerate(chunks):
            reps.append(s.step(n))
            if between is not None:
                between(i, s)
        return s.get_state(), reps


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_skip_equals_full_step_on_dry_start_floodplain(swe, prec):
    # dry start, inflow strip at the west edge: water spreads from there
    p = I.floodplain(384, 10.0, 2017, 2018, nsrc=20, hydro=I.Hydrograph(0, 5.0, 5.0, 3.0))
    p = p.to_f32_values() if prec == "f32" else p
    chunks = (1, 9, 20, 30)
    sa, ra = _run(swe, p, prec, chunks, skip=False)
    sb, rb = _run(swe, p, prec, chunks, skip=True)
    _same(sa, sb)
    _same_reports(ra, rb)
    assert all(r["skipped"] == 0 for r in ra)
    assert rb[-1]["skipped"] > 0 and rb[-1]["wet_cells"] > 0


def test_skip_matches_oracle_each_step_on_dry_start_floodplain(swe):
    """Skipping run against the FP64 oracle (not only against the run
    without skipping): dry-start 384^2 floodplain with a Gaussian inflow
    hydrograph at the west edge, FP64, skip on, 120 steps one at a time.
    Every step within 1e-12 relative L-inf of one oracle step from the
    GPU's own previous state (time, mass and wet cells likewise); the two
    trajectories within 1e-10 after 120 steps (one-step differences of
    1e-14 add up); most work items skipped throughout."""
    import oracle

    p = I.floodplain(384, 10.0, 2017, 2018, nsrc=20, hydro=I.Hydrograph(0, 5.0, 5.0, 3.0))
    bd = oracle._Bound(p)
    H, Qx, Qy, t = p.H, p.Qx, p.Qy, 0.0
    g = (H, Qx, Qy, t)
    skipped = []
    with swe.Solver.from_problem(p, "f64", seg_h=32, skip_dry=True) as s:
        for n in range(120):
            Hs, Qxs, Qys, info, _ = oracle.step(p, g[0], g[1], g[2], g[3], bound=bd)
            H, Qx, Qy, info_t, _ = oracle.step(p, H, Qx, Qy, t, bound=bd)
            t = info_t["t_new"]
            gi = s.step(1)
            g = s.get_state()
            assert abs(g[3] - info["t_new"]) <= 1e-13 * info["t_new"]
            for name, a, o in zip(("H", "Qx", "Qy"), g[:3], (Hs, Qxs, Qys)):
                err = np.abs(a - o).max() / max(np.abs(o).max(), 1e-6)
                assert err <= 1e-12, f"step {n + 1} {name}: rel Linf {err:.3e}"
            assert abs(gi["mass"] - info["mass"]) <= 1e-12 * max(info["mass"], 1e-300)
            assert gi["wet_cells"] == info["wet"]
            skipped.append(gi["skipped"])
    for name, a, o in zip(("H", "Qx", "Qy"), g[:3], (H, Qx, Qy)):
        err = np.abs(a - o).max() / max(np.abs(o).max(), 1e-6)
        assert err <= 1e-10, f"trajectory {name}: rel Linf {err:.3e}"
    assert abs(g[3] - t) <= 1e-12 * t
    assert info["wet"] > 0 and min(skipped[1:]) > 0


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_skip_with_gates_and_state_set_into_skipped_area(swe, prec):
    p = _patchy(300, 260, 51, prec, centre=(60, 70), radius=45)
    H, Qx, Qy = p.H.copy(), p.Qx.copy(), p.Qy.copy()
    # later, water is put into the far (skipped) corner through set_state
    H2 = H.copy()
    H2[200:230, 240:280] = 1.5
    gates = (np.array([60, 61, 62]), np.array([70, 70, 70]))

    def between(i, s):
        if i == 0:
            s.set_solid(gates[0], gates[1], np.ones(3, dtype=np.uint8))
        if i == 1:
            h, qx, qy, t = s.get_state()
            h = np.where(H2 != H, H2, h)
            s.set_state(h, qx, qy, t)
        if i == 2:
            s.set_solid(gates[0], gates[1], np.zeros(3, dtype=np.uint8))

    chunks = (6, 8, 8, 10)
    sa, ra = _run(swe, p, prec, chunks, skip=False, between=between)
    sb, rb = _run(swe, p, prec, chunks, skip=True, between=between)
    _same(sa, sb)
    _same_reports(ra, rb)
    assert min(r["skipped"] for r in rb) > 0


def test_skip_in_batched_ensemble(swe):
    probs = [_patchy(200 + 37 * s, 180 + 29 * s, 60 + s, "f32", centre=(50, 40), radius=35) for s in range(4)]
    ev = (np.array([0, 2, 2]), np.array([50, 45, 45]), np.array([40, 38, 38]), np.array([3, 2, 6]),
          np.array([1, 1, 0]))

    def run(skip):
        sols = [swe.Solver.from_problem(p, "f32", seg_h=32, skip_dry=skip) for p in probs]
        try:
            with swe.Batch(sols) as b:
                b.set_gate_events(*ev)
                r1 = b.step(4)
                r2 = b.step(8)
            return [x.get_state() for x in sols], r1 + r2
        finally:
            for x in sols:
                x.close()

    sa, ra = run(False)
    sb, rb = run(True)
    for x, y in zip(sa, sb):
        _same(x, y)
    _same_reports(ra, rb)
    assert all(r["skipped"] > 0 for r in rb)


def test_closed_steps_never_skip_but_keep_stamps(swe):
    # closed steps (learned closure attached) are computed in full; plain
    # steps after them still see the wet blocks the closed steps produced
    p = _patchy(192, 160, 77, "f32", centre=(50, 50), radius=30)
    from paper_1705_00614_gb300 import closure
    norm = closure.Norm(np.zeros(5), np.full(5, 5.0), np.zeros(3), np.full(3, 0.05))
    params = swe.flatten_cnn_params(closure.he_init(3))

    def run(skip):
        with swe.Solver.from_problem(p, "f32", seg_h=32, skip_dry=skip) as s, swe.CNN(1, 160, 192) as net:
            net.set_params(params)
            s.attach_closure(net, norm.all())
            r = [s.step_closed(5)]
            r.append(s.step(10))
            return s.get_state(), r

    sa, ra = run(False)
    sb, rb = run(True)
    _same(sa, sb)
    _same_reports(ra, rb)
    assert rb[0]["skipped"] == 0 and rb[1]["skipped"] > 0


def test_autotune_with_skipping_keeps_results(swe):
    # trial steps advance the stamps and the skip history; after the state is
    # restored nothing may rely on the buffer the trials wrote
    p = _patchy(280, 240, 91, "f32", centre=(70, 60), radius=40)
    sa, ra = _run(swe, p, "f32", (3, 12), skip=False)
    with swe.Solver.from_problem(p, "f32", seg_h=32, skip_dry=True) as s:
        s.autotune(3)
        rb = [s.step(3), s.step(12)]
        sb = s.get_state()
    _same(sa, sb)
    # the tiling may differ, so FP64 sums (mass, volumes) may be grouped
    # differently; everything else must agree exactly
    for x, y in zip(ra, rb):
        for k in ("t", "dt_last", "max_speed", "wet_cells", "step", "err_word"):
            assert x[k] == y[k], (k, x[k], y[k])
