"""Pins of the FP64 CNN-closure oracle (oracle/cnn_oracle.py): convolution
against SciPy's 2-D correlation, the exact adjoint identities of the data
and weight gradients, finite differences of the whole network's loss, Adam
against its closed form for a constant gradient, the 4x4 restriction's
conservation of block sums, and the closure's corrections: they act on
interior wet cells only, move no mass, and enter the oracle step's final
update as (tau/h) times their value."""
import numpy as np
import pytest
from scipy.signal import correlate2d

import oracle
from oracle import cnn_oracle as C
from paper_1705_00614_gb300 import inputs as I


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 9, 7, 3))
    w = rng.normal(size=(3, 3, 3, 4))
    b = rng.normal(size=4)
    y = C.conv3x3_fwd(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, :, :, c], w[:, :, c, o], mode="same", boundary="fill")
                             for c in range(3))
            assert np.allclose(y[n, :, :, o], ref, atol=1e-12)


def test_gradients_are_exact_adjoints():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 6, 8, 5))
    w = rng.normal(size=(3, 3, 5, 4))
    gy = rng.normal(size=(2, 6, 8, 4))
    y = C.conv3x3_fwd(x, w)
    gx = C.conv3x3_bwd_data(gy, w)
    gw, gb = C.conv3x3_bwd_weight(x, gy)
    lhs = np.sum(y * gy)
    assert abs(lhs - np.sum(x * gx)) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(w * gw)) < 1e-10 * abs(lhs)
    assert np.allclose(gb, gy.sum(axis=(0, 1, 2)))


def test_network_gradient_finite_differences():
    rng = np.random.default_rng(2)
    ch = (5, 6, 6, 3)
    params = C.init_params(3, ch)
    for l in range(len(params)):
        params[l][1] = rng.normal(0, 0.1, size=params[l][1].shape)
    x = rng.normal(size=(2, 5, 6, 5))
    t = rng.normal(size=(2, 5, 6, 3))

    def loss():
        return C.mse(C.forward(params, x)[-1], t)[0]

    acts = C.forward(params, x)
    _, gy = C.mse(acts[-1], t)
    grads = C.backward(params, acts, gy)
    h = 1e-6
    for l in range(len(params)):
        for k in range(2):
            flat = params[l][k].reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp = loss()
                flat[idx] = old - h
                lm = loss()
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[l][k].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (l, k, idx, fd, an)


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g, bias-corrected m = g and v = g^2 at every
    step, so each step moves a parameter by lr * g / (|g| + eps)."""
    p = [[np.array([1.0, -2.0]), np.array([0.5])]]
    g = [[np.array([0.3, -4.0]), np.array([2.0])]]
    m = [[np.zeros(2), np.zeros(1)]]
    v = [[np.zeros(2), np.zeros(1)]]
    for t in range(1, 6):
        C.adam(p, g, m, v, t, lr=0.01)
    step = 0.01 * g[0][0] / (np.abs(g[0][0]) + 1e-8)
    assert np.allclose(p[0][0], np.array([1.0, -2.0]) - 5 * step, atol=1e-12)


def test_restriction_conserves_block_sums():
    rng = np.random.default_rng(4)
    a = rng.normal(size=(3, 16, 24))
    r = C.restrict4(a)
    assert r.shape == (3, 4, 6)
    assert np.allclose(r.sum(axis=(1, 2)) * 16, a.sum(axis=(1, 2)))
    assert np.allclose(r[:, 1, 2], a[:, 4:8, 8:12].mean(axis=(1, 2)))


def test_bf16_rounding_definition():
    """Nearest bfloat16: exact on values with 8 significant bits, ties to
    even, relative error at most half an ulp, 2^-8."""
    assert C.round_bf16(1.0) == 1.0 and C.round_bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7
    assert C.round_bf16(1.0 + 2 ** -8) == 1.0            # tie -> even
    assert C.round_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie -> even (up)
    x = np.random.default_rng(8).normal(size=1000) * 1e3
    assert np.max(np.abs(C.round_bf16(x) - x) / np.abs(x)) <= 2 ** -8


def test_closure_corrections_move_no_mass_and_skip_shores():
    """Corrections act on cells >= 5 cm deep with four wet neighbours (not
    on the shore ring, a thin cell, or a cell at the grid edge), the depth
    part sums to zero over those cells, the momentum parts are the scaled
    network outputs there."""
    rng = np.random.default_rng(4)
    ny, nx = 12, 14
    H = np.full((ny, nx), 1.0)
    H[3:6, 4:8] = 0.0          # a dry island
    H[9, 9] = 0.03             # a thin cell
    y = rng.normal(size=(1, ny, nx, 3))
    mu, sd = np.array([0.5, -1.0, 2.0]), np.array([2.0, 3.0, 0.5])
    c = C.closure_corrections(y, H, 1e-4, mu, sd)
    on = C.correction_cells(H, 1e-4)
    assert not on[0].any() and not on[-1].any() and not on[:, 0].any() and not on[:, -1].any()
    assert not on[2:7, 3:9][H[2:7, 3:9] == 0.0].any() and not on[2, 5] and not on[6, 5] and not on[4, 3]
    assert not on[9, 9] and on[8, 9] and on[1, 1]  # the thin cell is still wet
    assert np.all(c[:, ~on] == 0.0)
    assert abs(c[0][on].sum()) <= 1e-12 * np.abs(c[0][on]).sum()
    for q in (1, 2):
        assert np.allclose(c[q][on], (y[0, ..., q] * sd[q] + mu[q])[on], rtol=0, atol=1e-15)


def test_oracle_step_applies_flux_corrections_in_the_final_update():
    """On a lake at rest over a flat bed every face flux is zero, so with
    corrections c the oracle's final update gives H = H0 + (tau/h) c_h and
    Q = (tau/h) c_v exactly where H stays wet: +c at one cell and -c at
    another leave the volume unchanged."""
    n, tau, dx = 16, 0.1, 2.0
    z = np.zeros((n, n))
    p = I.Problem("lake", I.Params(nx=n, ny=n, dx=dx, dt_fixed=tau), z.copy(), z.copy(), np.full((n, n), 1.5),
                  z.copy(), z.copy(), I.Sources.empty())
    corr = np.zeros((3, n, n))
    corr[0, 4, 5], corr[0, 10, 11] = 0.3, -0.3
    corr[1, 4, 5], corr[2, 10, 11] = 0.7, -0.2
    H, Qx, Qy, info, _ = oracle.step(p, p.H, p.Qx, p.Qy, 0.0, corr=corr)
    k = tau / dx
    assert H[4, 5] == 1.5 + k * 0.3 and H[10, 11] == 1.5 + k * -0.3
    assert Qx[4, 5] == k * 0.7 and Qy[10, 11] == k * -0.2
    mask = np.ones((n, n), bool)
    mask[4, 5] = mask[10, 11] = False
    assert np.all(H[mask] == 1.5) and np.all(Qx[mask] == 0.0) and np.all(Qy[mask] == 0.0)
    assert abs(info["mass"] - 1.5 * n * n * dx * dx) <= 1e-12 * info["mass"]


def test_bounded_corrections_are_clamped_to_a_fraction_of_the_flux_sums():
    """With a bound beta > 0 each correction c of a net flux sum f is applied
    as min(max(c, -beta |f|), beta |f|): on a lake at rest (every flux sum
    zero) no correction moves the water at all; on a dam break the change
    each bounded correction makes to H and Q is (tau/h) times the clamped
    value, with f read off the plain step (f = (new - post-Lagrangian) h/tau)."""
    rng = np.random.default_rng(11)
    beta = 0.5
    # lake at rest: all flux sums vanish, so every correction is clamped to 0
    n = 16
    z = np.zeros((n, n))
    lake = I.Problem("lake", I.Params(nx=n, ny=n, dx=2.0, dt_fixed=0.1), z.copy(), z.copy(), np.full((n, n), 1.5),
                     z.copy(), z.copy(), I.Sources.empty())
    corr = rng.normal(0.0, 5.0, size=(3, n, n))
    H, Qx, Qy, _, _ = oracle.step(lake, lake.H, lake.Qx, lake.Qy, 0.0, corr=corr, corr_bound=beta)
    assert np.all(H == 1.5) and np.all(Qx == 0.0) and np.all(Qy == 0.0)
    # dam break: compare with the plain step's flux sums
    p = I.dam_break(40, 1.0, 2.0, 1.0, ny=6)
    p.params.dt_fixed = 0.05
    Hp, Qxp, Qyp, info, st = oracle.step(p, p.H, p.Qx, p.Qy, 0.0, stages=True)
    k = info["tau"] / p.params.dx
    corr = rng.normal(0.0, 1.0, size=(3, 6, 40))
    Hb, Qxb, Qyb, _, _ = oracle.step(p, p.H, p.Qx, p.Qy, 0.0, corr=corr, corr_bound=beta)
    fh = (Hp - st["ht"]) / k
    fqx = (Qxp - st["qtx"]) / k
    for got, plain, f, c in ((Hb, Hp, fh, corr[0]), (Qxb, Qxp, fqx, corr[1])):
        lim = beta * np.abs(f)
        want = np.minimum(np.maximum(c, -lim), lim) * k
        assert np.abs((got - plain) - want).max() <= 1e-12
    clamped = np.abs(corr[0]) > beta * np.abs(fh)
    assert clamped.any() and (~clamped & (np.abs(fh) > 0)).any()
