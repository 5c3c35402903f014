"""Tensor-core (BF16, FP32 accumulation) CNN kernels against the FP64 CNN
oracle.  The kernels' inputs (images, BF16 weights) go to the oracle as the
same rounded values, and the oracle keeps hidden activations in BF16 as the
kernels do (cnn_oracle.round_bf16): then the forward output must agree
within 1e-2 and every parameter gradient within 2e-2 relative L2.  Against
the all-FP64 oracle the BF16 activations alone move the first layer's
weight gradient by ~2.2% (an oracle-side emulation shows the same number),
so that comparison is bounded by 3e-2.  Training lowers the loss."""
import numpy as np
import pytest

from oracle import cnn_oracle as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1705_00614_gb300 import build, swe
    build.build()
    swe.load()
    return torch, swe


def _bf16(torch, a):
    """Round to BF16 on the device; return (device tensor, FP64 numpy copy)."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16)
    return t, t.float().cpu().numpy().astype(np.float64)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _setup(torch, swe, n=2, h=32, w=48, seed=0):
    rng = np.random.default_rng(seed)
    params = C.init_params(seed)
    for l in range(4):
        params[l][1] = rng.normal(0, 0.05, size=params[l][1].shape)
    flat = swe.flatten_cnn_params(params)
    # the convolutions consume BF16 weights: give the oracle the same values
    params_r = swe.unflatten_cnn_params(flat)
    for l in range(4):
        params_r[l][0] = _bf16(torch, params_r[l][0])[1]
    x = np.zeros((n, h, w, 16))
    x[..., :5] = rng.normal(size=(n, h, w, 5))
    xd, x64 = _bf16(torch, x)
    t = rng.normal(size=(n, h, w, 3)).astype(np.float32)
    td = torch.from_numpy(t).cuda()
    return params_r, flat, xd, x64[..., :5], td, t.astype(np.float64)


# (n, h, w): narrower than one 128-pixel tile of the convolution kernel;
# one full plus one partial tile per row; then the work splits of real sizes
# on a 152-SM GPU (456 persistent convolution CTAs, up to 608 weight-gradient
# CTAs): 2 x 256 x 512 gives 416 items of 5 rows (the six-slot row ring
# wraps) and 2048 weight-gradient tiles (several per CTA); 1 x 1024 x 1024 is
# the 1024^2 coarse grid's own split (456 items of 18 rows, 8192 tiles); and
# 4 x 8 x 15360 makes 480 one-row-band items for 456 CTAs, so some CTAs run
# two items in a row.
SHAPES = [(2, 32, 48), (1, 16, 160), (2, 256, 512), (1, 1024, 1024), (4, 8, 15360)]


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(env, shape):
    torch, swe = env
    n, h, w = shape
    params, flat, xd, x64, td, t = _setup(torch, swe, n, h, w)
    with swe.CNN(n, h, w) as net:
        net.set_params(flat)
        y = torch.empty((n, h, w, 3), dtype=torch.float32, device="cuda")
        net.forward(xd.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        yg = y.cpu().numpy().astype(np.float64)
    yo = C.forward(params, x64)[-1]
    assert _rel(yg, yo) <= 1e-2


@pytest.mark.parametrize("shape", SHAPES)
def test_gradients_match_oracle(env, shape):
    torch, swe = env
    n, h, w = shape
    params, flat, xd, x64, td, t = _setup(torch, swe, n, h, w, seed=1)
    with swe.CNN(n, h, w) as net:
        net.set_params(flat)
        g, loss = net.gradients(xd.data_ptr(), td.data_ptr())
    gg = swe.unflatten_cnn_params(g)
    for store, tol in ((C.round_bf16, 2e-2), (None, 3e-2)):
        acts = C.forward(params, x64, store=store)
        lo, gy = C.mse(acts[-1], t)
        go = C.backward(params, acts, gy)
        assert abs(loss - lo) <= 1e-2 * lo
        for l in range(4):
            for k in range(2):
                err = _rel(gg[l][k], go[l][k])
                assert err <= tol, (store, l, k, err)


def test_training_lowers_the_loss(env):
    torch, swe = env
    params, flat, xd, x64, td, t = _setup(torch, swe, n=4, h=32, w=32, seed=2)
    # a learnable target: a fixed random network of the same shape applied to x
    teacher = C.init_params(9)
    t_np = C.forward(teacher, x64)[-1].astype(np.float32)
    td = torch.from_numpy(t_np).cuda()
    with swe.CNN(4, 32, 32) as net:
        net.set_params(flat)
        l0 = net.train_step(xd.data_ptr(), td.data_ptr(), 1e-3)
        for _ in range(300):
            l1 = net.train_step(xd.data_ptr(), td.data_ptr(), 1e-3, report=False)
        l1 = net.train_step(xd.data_ptr(), td.data_ptr(), 1e-3)
    assert l1 < 0.5 * l0, (l0, l1)
