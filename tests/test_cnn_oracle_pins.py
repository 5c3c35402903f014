"""Pins of the FP64 CNN-closure oracle (oracle/cnn_oracle.py): convolution
against SciPy's 2-D correlation, the exact adjoint identities of the data
and weight gradients, finite differences of the whole network's loss, Adam
against its closed form for a constant gradient, and the 4x4 restriction's
conservation of block sums."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn_oracle as C


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
