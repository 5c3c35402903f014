"""Pins of the FP64 oracle against what the mathematics fixes.

None of these compare the oracle with itself: each checks it against a
closed-form solution (Stoker, Ritter, Thacker, exact ODE solutions of single
force terms, the exact shallow-water Riemann solution), an exact invariant
(mass, lake at rest, y-invariance, x<->y symmetry) or a convergence order.
The paper prints no worked numbers, so these stand in for them; a plausible
slip anywhere in the oracle (a sign, a factor, a swapped index, a dropped
term) breaks at least one (see test_oracle_mutations.py).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1705_00614_gb300 import inputs as I
from tests import exact


def _box(n, H=1.0, ux=0.0, uy=0.0, manning=0.0, dx=1.0, **kw):
    z = np.zeros((n, n))
    p = I.Params(nx=n, ny=n, dx=dx, **kw)
    return I.Problem("box", p, z.copy(), np.full((n, n), manning), np.full((n, n), H),
                     np.full((n, n), H * ux), np.full((n, n), H * uy), I.Sources.empty())


def _centre_velocity(T, N, **kw):
    """Uniform flow in a box wide enough that the walls cannot reach the
    centre cell within N steps (dependence radius 6 cells per step)."""
    n = 2 * 6 * N + 9
    p = _box(n, **kw)
    p.params.dt_fixed = T / N
    H, Qx, Qy, t, _ = oracle.run(p, N)
    c = n // 2
    return Qx[c, c] / H[c, c], Qy[c, c] / H[c, c], t


def _orders(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


# ------------------------------------------------------------ dam breaks

def test_stoker_dam_break_256():
    """Wet dam break h_l = 2 m, h_r = 1 m, 256^2 cells, dx = 1 m, 200 steps,
    K = 0.3: against Stoker's solution at the final FP64 time."""
    p = I.dam_break(256, 1.0, 2.0, 1.0)
    H, Qx, Qy, t, infos = oracle.run(p, 200)
    # first step: the fastest signal is sqrt(g h_l) of the still left water
    assert abs(infos[0]["tau"] - 0.3 * 1.0 / math.sqrt(9.81 * 2.0)) < 1e-15
    xc = (np.arange(256) + 0.5)
    he, ue = exact.stoker(xc, t, 128.0, 2.0, 1.0)
    hm, um, S = exact.stoker_middle(2.0, 1.0)
    assert abs(hm - 1.4538) < 1e-3 and abs(S - 4.183) < 1e-3  # hand-checked values
    # mean depth error below 1% of the 1 m jump
    assert np.abs(H[0] - he).mean() < 0.01
    # bore position within 3 cells
    jump = 150 + int(np.argmax(-np.diff(H[0, 150:])))
    assert abs((jump + 1) - (128.0 + S * t)) < 3.0
    # plateau depth and velocity in the middle state
    mid = (xc > 128.0 + (um - math.sqrt(9.81 * hm)) * t + 5) & (xc < 128.0 + S * t - 5)
    assert mid.sum() > 10
    assert np.abs(H[0, mid] - hm).max() < 0.01 * hm
    assert np.abs(Qx[0, mid] / H[0, mid] - um).max() < 0.02 * um
    # the problem is y-invariant: all rows bitwise identical, no y momentum
    assert all(np.array_equal(H[j], H[0]) and np.array_equal(Qx[j], Qx[0]) for j in range(256))
    assert np.all(Qy == 0.0)
    # closed basin: mass constant to round-off
    m0 = 256 * (128 * 2.0 + 128 * 1.0)
    assert abs(infos[-1]["mass"] - m0) / m0 < 1e-13
    assert sum(i["clip_vol"] for i in infos) == 0.0


def test_stoker_converges():
    """L1 error of the wet dam break falls as the grid is refined."""
    errs = []
    for n, dx in ((128, 2.0), (256, 1.0), (512, 0.5)):
        p = I.dam_break(n, dx, 2.0, 1.0, x0=128.0, ny=4)
        p.params.dt_max = 10.0
        H, Qx, Qy, t, _ = oracle.run(p, 100000, t_end=10.0)
        assert abs(t - 10.0) < 1e-12
        xc = (np.arange(n) + 0.5) * dx
        he, _ = exact.stoker(xc, t, 128.0, 2.0, 1.0)
        errs.append(np.abs(H[1] - he).sum() * dx)
    assert errs[0] > errs[1] > errs[2]
    assert min(_orders(errs)) > 0.6  # first order at the bore


def test_ritter_dry_bed():
    """Dam break onto a dry bed (h_r = 0): the rarefaction fan of Ritter and
    a wet front that lags 2 c_l t by an amount that shrinks with dx."""
    lags, fan_errs = [], []
    for n, dx in ((128, 2.0), (256, 1.0), (512, 0.5)):
        p = I.dam_break(n, dx, 2.0, 0.0, x0=128.0, ny=4)
        H, Qx, Qy, t, infos = oracle.run(p, 100000, t_end=6.0)
        xc = (np.arange(n) + 0.5) * dx
        he, ue = exact.ritter(xc, t, 128.0, 2.0)
        cl = math.sqrt(9.81 * 2.0)
        fan = (xc > 128.0 - cl * t) & (xc < 128.0 + 1.0 * cl * t)
        fan_errs.append(np.abs(H[1, fan] - he[fan]).mean())
        front = (np.nonzero(H[1] > p.params.eps)[0].max() + 1) * dx
        lags.append(128.0 + 2.0 * cl * t - front)
        assert sum(i["clip_vol"] for i in infos) < 1e-12
    assert fan_errs[-1] < 0.01
    assert fan_errs[0] > fan_errs[1] > fan_errs[2]
    # the front is quantised to cells and slowed by the eps threshold: it
    # trails the exact one by a few percent and gets closer as dx shrinks
    cl = math.sqrt(9.81 * 2.0)
    assert 0.0 < lags[2] < lags[0] and lags[1] <= lags[0]
    assert lags[2] < 0.12 * 2.0 * cl * 6.0


# ------------------------------------------------------------ still water

def test_lake_at_rest_fractal_islands():
    """eta = 10 m over 0-30 m fractal terrain with dry islands, every force
    term on except wind: still water stays still to round-off."""
    p = I.lake_at_rest(96, 10.0, 7, eta0=10.0)
    wet = p.H > p.params.eps
    assert 0.02 < wet.mean() < 0.98 and (~wet).any()
    H, Qx, Qy, t, infos = oracle.run(p, 200)
    U = np.hypot(np.where(wet, Qx / np.where(wet, H, 1), 0), np.where(wet, Qy / np.where(wet, H, 1), 0))
    assert U.max() <= 1e-12
    assert np.abs((H + p.b) - (p.H + p.b))[wet].max() <= 1e-12
    assert np.abs(H - p.H)[~wet].max() == 0.0


def test_lake_at_rest_with_gates():
    """Closed gates are walls: still water around them stays still."""
    p = I.with_gates(I.lake_at_rest(64, 10.0, 11, eta0=15.0), 3, 6)
    p.solid[20:30, 31] = 1
    H, Qx, Qy, t, _ = oracle.run(p, 50)
    assert np.abs(Qx).max() <= 1e-12 and np.abs(Qy).max() <= 1e-12
    assert np.abs(H - p.H).max() <= 1e-12


# ------------------------------------------------------------ moving shoreline

@pytest.mark.parametrize("periods", [1])
def test_thacker_bowl(periods):
    """Planar oscillation in a paraboloid: L1 depth error after one period
    is small and falls with refinement."""
    errs = []
    for n in (64, 128):
        p = I.thacker_bowl(n)
        omega = math.sqrt(2 * 9.81 * 0.1)
        T = periods * 2 * math.pi / omega
        H, Qx, Qy, t, infos = oracle.run(p, 100000, t_end=T)
        assert abs(t - T) < 1e-12
        dx = 4.0 / n
        xc = -2 + (np.arange(n) + 0.5) * dx
        X, Y = np.meshgrid(xc, xc)
        He, ux, uy, _ = exact.thacker(X, Y, t)
        errs.append(np.abs(H - He).mean())
        m0, m1 = infos[0]["mass"] - infos[0]["src_vol"], infos[-1]["mass"]
        assert abs(m1 - oracle.mass(p, p.H)) < 1e-13 * m1
    assert errs[1] < errs[0]
    assert errs[1] < 0.03 * 0.125  # 3% of the largest depth


# ------------------------------------------------------------ single force terms

def test_coriolis_inertial_rotation_second_order():
    """Uniform flow, Coriolis only: U turns clockwise by f t (northern
    hemisphere); the predictor-corrector converges at second order."""
    f, T = 0.1, 10.0
    errs = []
    for N in (4, 8, 16):
        ux, uy, t = _centre_velocity(T, N, ux=1.0, uy=0.5, coriolis_f=f)
        th = -f * t
        ex = (math.cos(th) * 1.0 - math.sin(th) * 0.5, math.sin(th) * 1.0 + math.cos(th) * 0.5)
        errs.append(math.hypot(ux - ex[0], uy - ex[1]))
    assert all(1.9 < o < 2.1 for o in _orders(errs))
    assert errs[-1] < 1e-3


def test_friction_decay_matches_manning_ode():
    """Uniform flow, Manning friction only: U' = -g n^2 U|U| / H^{4/3} has
    U = U0 / (1 + g n^2 U0 t / H^{4/3}); the point-implicit friction
    converges to it at first order."""
    g, nM, U0, H = 9.81, 0.05, 2.0, 1.5
    errs = []
    for N in (4, 8, 16):
        ux, uy, t = _centre_velocity(40.0, N, ux=U0, H=H, manning=nM)
        ex = U0 / (1.0 + g * nM * nM * U0 * t / H ** (4.0 / 3.0))
        errs.append(abs(ux - ex))
        assert uy == 0.0
    assert all(0.9 < o < 1.3 for o in _orders(errs))
    assert errs[-1] < 0.02 * U0


def test_wind_spin_up_second_order():
    """Still shallow water under a uniform wind: v = W - U obeys
    v' = -C_a (rho_a/rho) v|v| / H, so v = W / (1 + C_a (rho_a/rho) W t / H)."""
    ca, ra, W, H = 1.3e-3, 1.225e-3, 20.0, 0.05
    k = ca * ra
    errs = []
    for N in (4, 8, 16):
        ux, uy, t = _centre_velocity(60.0, N, H=H, wind_x=W, c_a=ca, rho_air_over_rho=ra)
        errs.append(abs(ux - (W - W / (1.0 + k * W * t / H))))
    assert all(1.9 < o < 2.1 for o in _orders(errs))


def test_viscous_shear_mode_decay():
    """U_x = A cos(pi m (j + 1/2) / N) is an eigenmode of the 5-point
    Laplacian with no-stress walls; it decays at the discrete rate
    lambda = nu (2 - 2 cos(pi m / N)) / h^2, approached at second order in
    tau, and lambda tends to nu (pi m / L)^2."""
    nu, ny, m, A, h = 2.0, 32, 2, 0.1, 2.0
    T = 8.0
    lam = nu * (2.0 - 2.0 * math.cos(math.pi * m / ny)) / (h * h)
    errs = []
    for N in (4, 8, 16):
        nx = 2 * 6 * N + 9
        z = np.zeros((ny, nx))
        jj = (np.arange(ny) + 0.5)
        ux = A * np.cos(math.pi * m * jj / ny)[:, None] * np.ones((1, nx))
        p = I.Params(nx=nx, ny=ny, dx=h, nu=nu, dt_fixed=T / N)
        prob = I.Problem("shear", p, z.copy(), z.copy(), np.ones((ny, nx)), ux.copy(), z.copy(),
                         I.Sources.empty())
        H, Qx, Qy, t, _ = oracle.run(prob, N)
        c = nx // 2
        errs.append(np.abs(Qx[:, c] / H[:, c] - ux[:, c] * math.exp(-lam * t)).max())
    assert all(1.9 < o < 2.1 for o in _orders(errs))
    assert abs(lam / (nu * (math.pi * m / (ny * h)) ** 2) - 1.0) < 0.01


def test_tvd_transverse_velocity_advection():
    """U_y(x) is a step profile carried by a uniform U_x on flat water: the
    momentum flux is MUSCL-minmod upwinding, a TVD scheme at this Courant
    number (Harten 1983), so no new extrema may appear while the step moves
    downstream."""
    nx, ny = 120, 40
    z = np.zeros((ny, nx))
    uy = np.where((np.arange(nx) >= 30) & (np.arange(nx) < 50), 0.02, -0.01)[None, :].repeat(ny, 0)
    p = I.Params(nx=nx, ny=ny, dx=1.0)
    prob = I.Problem("tvd", p, z.copy(), z.copy(), np.ones((ny, nx)), np.ones((ny, nx)), uy.copy(),
                     I.Sources.empty())
    H, Qx, Qy, t, _ = oracle.run(prob, 40)
    v = Qy[ny // 2, 10:nx - 30] / H[ny // 2, 10:nx - 30]
    assert v.max() <= 0.02 + 1e-12 and v.min() >= -0.01 - 1e-12
    # the step did move: the profile is no longer the initial one
    assert np.abs(v - uy[ny // 2, 10:nx - 30]).max() > 1e-3


def test_drain_on_dry_ground_removes_nothing():
    """A drain (sigma < 0) on a dry cell has no water to take: volume
    unchanged, nothing clipped, zero source volume."""
    p = I.lake_at_rest(48, 10.0, 13, eta0=12.0)
    dry = np.argwhere(p.H <= p.params.eps)
    wet = np.argwhere(p.H > 1.0)
    assert len(dry) > 4 and len(wet) > 4
    iy = np.array([dry[0][0], dry[1][0], wet[0][0]], dtype=np.int32)
    ix = np.array([dry[0][1], dry[1][1], wet[0][1]], dtype=np.int32)
    z = np.zeros(3)
    src = I.Sources(ix, iy, np.array([1.0, 1.0, 0.0]), z, z, np.zeros(3, dtype=np.int32),
                    [I.Hydrograph(1, -0.5)])
    prob = I.Problem("drain", p.params, p.b, p.n_manning, p.H, p.Qx, p.Qy, src)
    m0 = oracle.mass(prob, p.H)
    H, Qx, Qy, t, infos = oracle.run(prob, 10)
    assert sum(i["src_vol"] for i in infos) == 0.0
    assert sum(i["clip_vol"] for i in infos) == 0.0
    assert abs(infos[-1]["mass"] - m0) <= 1e-13 * m0



def test_drain_emptying_a_moving_cell_leaves_no_momentum():
    """A drain that takes more than a moving cell holds (H + tau sigma < 0)
    empties it: no water is left to carry momentum, so the post-Lagrangian
    momentum is zero, and the water the face fluxes then bring in (from the
    west and from the east, both carrying the +x flow) gives the cell
    positive x momentum, never the reversed momentum of a negative depth."""
    n, c = 24, 12
    p = _box(n, H=0.1, ux=1.0, dx=1.0, dt_fixed=0.05)
    src = I.Sources(np.array([c], dtype=np.int32), np.array([c], dtype=np.int32), np.array([1.0]),
                    np.zeros(1), np.zeros(1), np.zeros(1, dtype=np.int32), [I.Hydrograph(1, -20.0)])
    prob = I.Problem("drain", p.params, p.b, p.n_manning, p.H, p.Qx, p.Qy, src)
    Hn, Qxn, Qyn, info, st = oracle.step(prob, p.H, p.Qx, p.Qy, 0.0, stages=True)
    assert st["utx"][c, c] > 0.9  # the water that was there moved at about +1 m/s
    assert st["ht"][c, c] == 0.0 and st["qtx"][c, c] == 0.0 and st["qty"][c, c] == 0.0
    assert Hn[c, c] > prob.params.eps  # refilled by the face fluxes
    assert Qxn[c, c] > 0.0 and Qxn[c, c] / Hn[c, c] <= 1.0 + 1e-12
    assert abs(Qyn[c, c]) <= 1e-15
    # the drain removed exactly the 0.1 m the cell held
    assert abs(info["src_vol"] - (-0.1)) <= 1e-15


# ------------------------------------------------------------ signal speed

def _wind_box(u, w, H=0.01, dx=4.0, n=12):
    """Uniform flow U on a flat frictionless bed under wind W.  The pressure
    and viscous terms vanish for a uniform state, Coriolis is off, so the
    acceleration is the wind stress alone: a = C_a (rho_a/rho) (W - U)|W - U| / H."""
    return _box(n, H=H, ux=u[0], uy=u[1], dx=dx, wind_x=w[0], wind_y=w[1], c_a=1.0,
                rho_air_over_rho=1.0e-3, coriolis_f=0.0, nu=0.0, cfl=0.3, dt_max=10.0)


@pytest.mark.parametrize("u,w", [((3.0, 0.0), (-20.0, 0.0)),   # a against U along x
                                 ((0.0, 3.0), (0.0, -20.0)),   # the same along y
                                 ((3.0, 0.0), (30.0, 0.0)),    # a along U
                                 ((-2.0, 1.0), (15.0, -25.0))])  # both components
def test_time_step_from_particle_speed(u, w):
    """Where the acceleration is strong and the layer thin, the particle
    speed U_p = max_d |U_d + sgn(a_d) sqrt(h |a_d|)| exceeds the wave speed
    U_s = max(|U_x|, |U_y|) + sqrt(g H) and sets tau = K h / max(U_s, U_p)
    (Sec. 2.3, Fig. 2).  Here a is known in closed form (wind stress only)."""
    H, dx, g, K = 0.01, 4.0, 9.81, 0.3
    p = _wind_box(u, w, H=H, dx=dx)
    dwx, dwy = w[0] - u[0], w[1] - u[1]
    wm = math.hypot(dwx, dwy)
    a = (1.0e-3 * dwx * wm / H, 1.0e-3 * dwy * wm / H)
    us = max(abs(u[0]), abs(u[1])) + math.sqrt(g * H)
    up = max(abs(u[d] + math.copysign(math.sqrt(dx * abs(a[d])), a[d])) if a[d] != 0.0 else abs(u[d])
             for d in range(2))
    assert up > 1.2 * us  # the case really is set by the particle speed
    _, _, _, info, _ = oracle.step(p, p.H, p.Qx, p.Qy, 0.0)
    assert abs(info["smax"] - up) <= 1e-14 * up
    assert abs(info["tau"] - K * dx / up) <= 1e-14 * (K * dx / up)


def test_time_step_from_wave_speed_two_components():
    """A deep uniform flow with both components nonzero and no force (no
    wind stress since W = U, flat bed): a = 0, so U_p = max(|U_x|, |U_y|)
    and the wave speed U_s = max(|U_x|, |U_y|) + sqrt(g H) sets
    tau = K h / U_s (Sec. 2.3, Fig. 2)."""
    u, H, dx, g, K = (3.0, -4.0), 2.0, 4.0, 9.81, 0.3
    p = _wind_box(u, u, H=H, dx=dx)
    us = max(abs(u[0]), abs(u[1])) + math.sqrt(g * H)
    _, _, _, info, _ = oracle.step(p, p.H, p.Qx, p.Qy, 0.0)
    assert abs(info["smax"] - us) <= 1e-14 * us
    assert abs(info["tau"] - K * dx / us) <= 1e-14 * (K * dx / us)


# ------------------------------------------------------------ Riemann solver

def test_riemann_two_rarefactions_is_exact():
    """When both waves are rarefactions the two-rarefaction solver is the
    exact solution, so it must agree with an exact iterative solver."""
    rng = np.random.default_rng(3)
    n = 0
    while n < 200:
        hl, hr = rng.uniform(0.1, 5.0, 2)
        ul, ur = rng.uniform(-3, 3, 2)
        ur = ul + rng.uniform(0.05, 2.0 * (math.sqrt(9.81 * hl) + math.sqrt(9.81 * hr)) - 0.1)
        cs = 0.5 * (math.sqrt(9.81 * hl) + math.sqrt(9.81 * hr)) + 0.25 * (ul - ur)
        hs = cs * cs / 9.81
        if not (hs < hl and hs < hr):
            continue
        n += 1
        h, u = oracle.riemann(9.81, 1e-4, hl, ul, hr, ur)
        he, ue = exact.exact_riemann_face(hl, ul, hr, ur)
        assert abs(h - he) < 1e-10 * max(1.0, he) and abs(u - ue) < 1e-10 * max(1.0, abs(ue))


def test_riemann_shock_cases_close_to_exact():
    """With shocks the solver is approximate: mass flux within 5% of the
    exact one (relative to sqrt(g h) h), and exact for equal states."""
    rng = np.random.default_rng(4)
    for _ in range(200):
        hl, hr = rng.uniform(0.5, 3.0, 2)
        ul, ur = rng.uniform(-1.0, 1.0, 2)
        h, u = oracle.riemann(9.81, 1e-4, hl, ul, hr, ur)
        he, ue = exact.exact_riemann_face(hl, ul, hr, ur)
        scale = max(hl, hr) * math.sqrt(9.81 * max(hl, hr))
        assert abs(h * u - he * ue) < 0.05 * scale
    for hh, uu in ((1.0, 0.3), (2.0, -0.7), (0.5, 5.0), (0.5, -5.0)):
        h, u = oracle.riemann(9.81, 1e-4, hh, uu, hh, uu)
        assert abs(h - hh) < 1e-14 and abs(u - uu) < 1e-14


def test_riemann_dry_bed_fan_and_mirror():
    """Dry right side: the face sits in Ritter's fan, h = (u_l + 2 c_l)^2 /
    (9 g), u = (u_l + 2 c_l) / 3.  Mirroring the problem mirrors the answer."""
    g = 9.81
    for hl, ul in ((1.0, 0.0), (2.0, 1.0), (0.3, -0.5)):
        cl = math.sqrt(g * hl)
        h, u = oracle.riemann(g, 1e-4, hl, ul, 0.0, 0.0)
        assert abs(h - (ul + 2 * cl) ** 2 / (9 * g)) < 1e-14
        assert abs(u - (ul + 2 * cl) / 3) < 1e-14
    h, u = oracle.riemann(g, 1e-4, 1.0, -7.0, 0.0, 0.0)  # front u_l + 2 c_l < 0: face dry
    assert h == 0.0 and u == 0.0
    rng = np.random.default_rng(5)
    for _ in range(100):
        hl, hr = rng.uniform(0, 3, 2)
        ul, ur = rng.uniform(-4, 4, 2)
        h1, u1 = oracle.riemann(g, 1e-4, hl, ul, hr, ur)
        h2, u2 = oracle.riemann(g, 1e-4, hr, -ur, hl, -ul)
        assert abs(h1 - h2) < 1e-13 and abs(u1 + u2) < 1e-13


# ------------------------------------------------------------ invariants

def test_transpose_symmetry_random_wet_dry():
    """Swapping x and y in every input (wind components swapped, Coriolis
    sign flipped since the swap is a reflection) swaps the outputs."""
    p = I.random_wet_dry(40, 28, seed=21)
    T = I.Problem("t", I.Params(**{**p.params.__dict__, "nx": 28, "ny": 40,
                                   "wind_x": p.params.wind_y, "wind_y": p.params.wind_x,
                                   "coriolis_f": -p.params.coriolis_f}),
                  p.b.T.copy(), p.n_manning.T.copy(), p.H.T.copy(), p.Qy.T.copy(), p.Qx.T.copy(),
                  I.Sources(p.sources.iy, p.sources.ix, p.sources.weight, p.sources.vy,
                            p.sources.vx, p.sources.hydro, p.sources.hydrographs))
    H1, Qx1, Qy1, t1, _ = oracle.run(p, 5)
    H2, Qx2, Qy2, t2, _ = oracle.run(T, 5)
    assert abs(t1 - t2) < 1e-13
    for a, b in ((H1, H2.T), (Qx1, Qy2.T), (Qy1, Qx2.T)):
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())


def test_closed_basin_mass_all_physics():
    """Random wet/dry state, every force on, no sources: mass constant to
    FP64 round-off and no negative depths clipped."""
    p = I.random_wet_dry(48, 40, seed=5, with_sources=False)
    m0 = oracle.mass(p, p.H)
    H, Qx, Qy, t, infos = oracle.run(p, 60)
    clip = sum(i["clip_vol"] for i in infos)
    assert abs(infos[-1]["mass"] - clip - m0) <= 1e-13 * m0
    assert np.all(H >= 0.0)


def test_source_volume_matches_hydrograph_integral():
    """Sources on dry cells: the injected volume equals h^2 * weight * the
    integral of the Gaussian hydrograph (erf closed form) up to the
    midpoint-rule error, and the mass budget closes to round-off."""
    p = I.floodplain(96, 10.0, 31, 32, nsrc=20, hydro=I.Hydrograph(0, 5.0, 30.0, 10.0))
    H, Qx, Qy, t, infos = oracle.run(p, 100000, t_end=60.0)
    vol = sum(i["src_vol"] for i in infos)
    s, tp, peak = 10.0, 30.0, 5.0
    integral = peak * s * math.sqrt(math.pi / 2) * (math.erf((60 - tp) / (s * math.sqrt(2)))
                                                   - math.erf((0 - tp) / (s * math.sqrt(2))))
    assert abs(vol - integral * 100.0) < 2e-3 * integral * 100.0
    clip = sum(i["clip_vol"] for i in infos)
    assert abs(infos[-1]["mass"] - vol - clip) <= 1e-12 * infos[-1]["mass"]


def test_y_invariant_dam_break_keeps_rows_identical():
    """A dam break along x is the same in every row: after many steps all
    rows are bitwise equal and the y momentum is exactly zero (the wall
    rows see no y pressure difference and every y face carries no flux)."""
    p = I.dam_break(64, 1.0, 2.0, 1.0, ny=24)
    H, Qx, Qy, t, _ = oracle.run(p, 80)
    for a in (H, Qx):
        assert np.array_equal(a, np.repeat(a[:1], a.shape[0], axis=0))
    assert not Qy.any()
    assert H[0].max() < 2.0 and H[0].min() > 1.0  # the waves have moved
