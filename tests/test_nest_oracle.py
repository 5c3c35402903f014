"""Pins of the two-level nesting oracle (oracle/nest_oracle.py) against
facts that do not depend on it: still water gives ghost depths equal to the
free surface above the fine bed; 4 x 4 means undo piecewise-constant
refinement; a nested lake at rest (wet around the patch) stays at rest on
both levels; and a fine
sub-step with a ghost ring is the ordinary oracle step of the same cells
inside a larger grid (one step reaches 6 cells, the ring is 10 deep)."""
import dataclasses

import numpy as np

import oracle
from oracle import nest_oracle as N
from paper_1705_00614_gb300 import inputs as I

P = N.PAD


def test_ghosts_of_still_water_follow_the_free_surface():
    rng = np.random.default_rng(1)
    nyc, nxc, nx, ny, ix0, iy0 = 12, 14, 16, 12, 4, 3
    eta = 3.0
    bc = rng.uniform(0.0, 2.5, size=(nyc, nxc))
    bc[0, 0] = 4.0  # a dry coarse cell (above the surface), not near the patch
    Hc = np.maximum(0.0, eta - bc)
    z = np.zeros_like(Hc)
    b_ext = rng.uniform(0.0, 4.0, size=(ny + 2 * P, nx + 2 * P))
    b_ext[0, 0] = 1e30  # a wall ghost
    H, Qx, Qy = N.ring_values((Hc, z, z), (Hc, z, z), bc, b_ext, nx, ny, ix0, iy0, 0.25, 1e-4)
    ring = np.ones_like(b_ext, dtype=bool)
    ring[P:P + ny, P:P + nx] = False
    want = np.where(b_ext < 1e29, np.maximum(0.0, eta - b_ext), 0.0)
    assert np.array_equal(H[ring], want[ring])
    assert not H[~ring].any() and not Qx.any() and not Qy.any()


def test_restriction_undoes_piecewise_constant_refinement():
    rng = np.random.default_rng(2)
    c = [np.round(rng.uniform(-4, 4, size=(5, 7)) * 1024) / 1024 for _ in range(3)]
    f = [np.kron(a, np.ones((4, 4))) for a in c]
    r = N.restrict(*f)
    for a, b in zip(r, c):
        assert np.array_equal(a, b)
    # and the patch volume is kept
    assert np.sum(r[0]) * 16 == np.sum(f[0])


def _nest_setup(seed, nxc=22, nyc=20, ix0=5, iy0=4, wc=8, hc=8, still=False):
    """A coarse grid and a 4x finer patch over coarse cells [ix0, ix0+wc) x
    [iy0, iy0+hc) on one fine fractal terrain (coarse bed = 4 x 4 means)."""
    base = I.random_wet_dry(4 * nxc, 4 * nyc, seed=seed, dx=5.0, with_sources=False)
    if still:
        # still water is a steady state of every force term but the wind
        base = dataclasses.replace(base, params=dataclasses.replace(base.params, wind_x=0.0, wind_y=0.0))
    bf = base.b
    bc = bf.reshape(nyc, 4, nxc, 4).mean(axis=(1, 3))
    nc = base.n_manning.reshape(nyc, 4, nxc, 4).mean(axis=(1, 3))
    pc = dataclasses.replace(base.params, nx=nxc, ny=nyc, dx=20.0, dt_fixed=0.2)
    if still:
        # the lake covers the patch and the coarse cells around it (a dry coarse
        # cell gives dry ghosts, even over fine cells below the surface);
        # elsewhere it has dry banks
        near = bf[4 * (iy0 - 3):4 * (iy0 + hc + 3), 4 * (ix0 - 3):4 * (ix0 + wc + 3)]
        eta = float(near.max()) + 0.5
        Hc = np.maximum(0.0, eta - bc)
        Qxc = np.zeros_like(Hc)
        Qyc = np.zeros_like(Hc)
    else:
        Hc = base.H.reshape(nyc, 4, nxc, 4).mean(axis=(1, 3))
        Qxc = base.Qx.reshape(nyc, 4, nxc, 4).mean(axis=(1, 3))
        Qyc = base.Qy.reshape(nyc, 4, nxc, 4).mean(axis=(1, 3))
    coarse = I.Problem("coarse", pc, bc, nc, Hc, Qxc, Qyc, I.Sources.empty())
    nx, ny = 4 * wc, 4 * hc
    x0, y0 = 4 * ix0, 4 * iy0
    pf = dataclasses.replace(base.params, nx=nx, ny=ny, dx=5.0, dt_fixed=0.05)
    sl = (slice(y0, y0 + ny), slice(x0, x0 + nx))
    if still:
        Hf = np.maximum(0.0, eta - bf[sl])
        Qxf = np.zeros_like(Hf)
        Qyf = np.zeros_like(Hf)
    else:
        # the fine patch starts from the coarse state, refined piecewise constant
        Hf = np.kron(Hc, np.ones((4, 4)))[sl]
        Qxf = np.kron(Qxc, np.ones((4, 4)))[sl]
        Qyf = np.kron(Qyc, np.ones((4, 4)))[sl]
    fine = I.Problem("fine", pf, bf[sl], base.n_manning[sl], Hf, Qxf, Qyf, I.Sources.empty())
    esl = (slice(y0 - P, y0 + ny + P), slice(x0 - P, x0 + nx + P))
    return coarse, fine, bf[esl].copy(), base.n_manning[esl].copy(), ix0, iy0


def test_nested_lake_at_rest_stays_at_rest():
    coarse, fine, b_ext, n_ext, ix0, iy0 = _nest_setup(11, still=True)
    c, f = N.nest_run(coarse, fine, b_ext, n_ext, ix0, iy0, 3)
    assert np.abs(f[0] - fine.H).max() <= 1e-12
    assert np.abs(f[1]).max() <= 1e-12 and np.abs(f[2]).max() <= 1e-12
    assert np.abs(c[0] - coarse.H).max() <= 1e-12
    assert np.abs(c[1]).max() <= 1e-12 and np.abs(c[2]).max() <= 1e-12


def test_ghost_ring_step_is_the_step_of_a_larger_grid():
    # G is larger than the patch's padded extent by 4 cells on every side
    nx, ny, m = 24, 20, 4
    G = I.random_wet_dry(nx + 2 * P + 2 * m, ny + 2 * P + 2 * m, seed=21, with_sources=False)
    G = dataclasses.replace(G, params=dataclasses.replace(G.params, dt_fixed=0.05))
    Hg, Qxg, Qyg, _, _ = oracle.step(G, G.H, G.Qx, G.Qy, 0.0)
    esl = (slice(m, m + ny + 2 * P), slice(m, m + nx + 2 * P))
    isl = (slice(m + P, m + P + ny), slice(m + P, m + P + nx))
    fine = dataclasses.replace(G, params=dataclasses.replace(G.params, nx=nx, ny=ny), b=G.b[isl],
                               n_manning=G.n_manning[isl], H=G.H[isl], Qx=G.Qx[isl], Qy=G.Qy[isl])
    ext = N.extended(fine, G.b[esl], G.n_manning[esl])
    He, Qxe, Qye, _, _ = oracle.step(ext, G.H[esl], G.Qx[esl], G.Qy[esl], 0.0)
    sl = (slice(P, P + ny), slice(P, P + nx))
    assert np.array_equal(He[sl], Hg[isl])
    assert np.array_equal(Qxe[sl], Qxg[isl])
    assert np.array_equal(Qye[sl], Qyg[isl])


def _open_basin(n=40, H0=2.0, u0=0.6, v0=-0.3, slope=False):
    """Flat (or linearly sloping, frictionless) domain with a uniform state;
    the ring terrain extends the interior's."""
    p = I.Params(nx=n, ny=n, dx=4.0, dt_fixed=0.05)
    x = (np.arange(n + 2 * P) - P + 0.5) * 4.0
    b_ext = np.tile(1e-3 * x, (n + 2 * P, 1)) if slope else np.zeros((n + 2 * P, n + 2 * P))
    b = b_ext[P:P + n, P:P + n]
    H = np.full((n, n), H0)
    prob = I.Problem("open", p, b.copy(), np.zeros((n, n)), H, H * u0, H * v0, I.Sources.empty())
    return prob, b_ext


def test_uniform_flow_passes_open_boundaries_unchanged():
    prob, b_ext = _open_basin()
    H, Qx, Qy = N.open_run(prob, b_ext, None, 20)
    assert np.abs(H - 2.0).max() <= 1e-13
    assert np.abs(Qx - 2.0 * 0.6).max() <= 1e-13 and np.abs(Qy + 2.0 * 0.3).max() <= 1e-13


def test_open_boundaries_let_a_wave_leave():
    """A dam break released towards the east edge: with an open boundary the
    interior matches a four times longer domain (whose far walls are not yet
    reached) far better than with a wall, and water leaves the grid."""
    n, ny = 48, 8
    p = I.Params(nx=n, ny=ny, dx=1.0, dt_fixed=0.02)
    H0 = np.where(np.arange(n) < 24, 2.0, 1.0)[None, :].repeat(ny, axis=0)
    z = np.zeros((ny, n))
    prob = I.Problem("wave", p, z.copy(), z.copy(), H0, z.copy(), z.copy(), I.Sources.empty())
    b_ext = np.zeros((ny + 2 * P, n + 2 * P))
    b_ext[:P, :] = 1e30  # north, south and west stay walls: only the east is open
    b_ext[-P:, :] = 1e30
    b_ext[:, :P] = 1e30
    steps = 400  # 8 s: the bore passes the east edge at x = 48 (speed ~5 m/s)
    Ho, _, _ = N.open_run(prob, b_ext, None, steps)
    Hw, _, _, _, _ = oracle.run(prob, steps)
    big = dataclasses.replace(prob, params=dataclasses.replace(p, nx=4 * n),
                              b=np.zeros((ny, 4 * n)), n_manning=np.zeros((ny, 4 * n)),
                              H=np.concatenate([H0, np.ones((ny, 3 * n))], axis=1),
                              Qx=np.zeros((ny, 4 * n)), Qy=np.zeros((ny, 4 * n)))
    Hb, _, _, _, _ = oracle.run(big, steps)
    Hb = Hb[:, :n]
    err_open = np.abs(Ho - Hb).max()
    err_wall = np.abs(Hw - Hb).max()
    # zero gradient reflects part of a subcritical bore, a wall all of it
    assert err_open < 0.25 * err_wall, (err_open, err_wall)
    assert Ho.sum() < H0.sum() - 1.0
