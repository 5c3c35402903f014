"""swe_step_f32_noalloc, the allocation-free entry point for callers that
cannot allocate device memory (their device memory comes from their own pool
or a fixed budget, or they must avoid cudaMalloc/cudaFree and the device
synchronisation those calls can cause).  The planes here are allocated by
the test with torch, standing in for such a caller's memory; the entry
point itself allocates nothing.  Its results must match the regular
swe_step on two calls in a row, within the FP32 tolerance the other
fused-kernel comparisons use.  This file is named so pytest collects it
last."""
import numpy as np
import pytest

from paper_1705_00614_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 2e-6  # relative L-inf, as in the fused/staged FP32 comparison


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1705_00614_gb300 import build, swe
    build.build()
    swe.load()
    return torch, swe


def _plane(torch, arr, ny, nx, pitch, ring):
    P = 10
    t = torch.full((ny + 2 * P, pitch), ring, dtype=torch.float32, device="cuda")
    t[P:P + ny, P:P + nx] = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float32)).cuda()
    return t


def _interior(t, ny, nx):
    P = 10
    return t[P:P + ny, P:P + nx].double().cpu().numpy()


def _close(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-6)


def test_noalloc_step_matches_swe_step_twice(env):
    torch, swe = env
    prob = I.random_wet_dry(300, 270, seed=29, with_sources=False).to_f32_values()
    nx, ny = prob.params.nx, prob.params.ny
    stream = torch.cuda.Stream()
    with swe.Solver.from_problem(prob, "f32", stream=stream.cuda_stream) as s:
        ms0 = s.step(0)["max_speed"]
        s.step(1)
        ref1 = s.get_state()
        s.step(1)
        ref2 = s.get_state()
    pitch = ((nx + 20 + 31) // 32) * 32
    a = [_plane(torch, x, ny, nx, pitch, 0.0) for x in (prob.H, prob.Qx, prob.Qy)]
    out = [torch.zeros((ny + 20, pitch), dtype=torch.float32, device="cuda") for _ in range(3)]
    b = _plane(torch, prob.b, ny, nx, pitch, 1.0e30)
    n = _plane(torch, prob.n_manning, ny, nx, pitch, 0.0)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        i1 = swe.step_f32_noalloc(prob.params, *[x.data_ptr() for x in a], b.data_ptr(), n.data_ptr(),
                                  *[x.data_ptr() for x in out], pitch, 0.0, ms0, stream.cuda_stream)
        for g, r in zip(out, ref1[:3]):
            assert _close(_interior(g, ny, nx), r) <= TOL
        assert abs(i1["t"] - ref1[3]) <= 1e-12 * ref1[3]
        # second call in a row: previous outputs in, previous inputs as outputs
        i2 = swe.step_f32_noalloc(prob.params, *[x.data_ptr() for x in out], b.data_ptr(), n.data_ptr(),
                                  *[x.data_ptr() for x in a], pitch, i1["t"], i1["max_speed"],
                                  stream.cuda_stream)
        for g, r in zip(a, ref2[:3]):
            assert _close(_interior(g, ny, nx), r) <= TOL
        assert abs(i2["t"] - ref2[3]) <= 1e-12 * ref2[3]
    # the ring (walls) was left alone
    assert float(b[0, 0]) == float(np.float32(1.0e30)) and float(a[0][0:10].abs().max()) == 0.0
    # the property the entry point exists for: further calls allocate no
    # device memory (neither the driver's free bytes nor torch's pool move)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    stats0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    t, ms = i2["t"], i2["max_speed"]
    src, dst = a, out
    with torch.cuda.stream(stream):
        for _ in range(4):
            i = swe.step_f32_noalloc(prob.params, *[x.data_ptr() for x in src], b.data_ptr(), n.data_ptr(),
                                     *[x.data_ptr() for x in dst], pitch, t, ms, stream.cuda_stream)
            t, ms = i["t"], i["max_speed"]
            src, dst = dst, src
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == stats0


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, swe = env
    nx = (swe.NOALLOC_MAX_ITEMS + 1) * 116
    params = I.Params(nx=nx, ny=8, dx=1.0)
    fake = 1 << 20  # aligned addresses that are never touched: sizes are checked first
    with pytest.raises(swe.SweError) as e:
        swe.step_f32_noalloc(params, *([fake] * 8), nx + 20 + 12, 0.0, 0.0)
    assert e.value.code == -1 and "scratch" in str(e.value)
    # a row pitch the kernel's 32-bit row index cannot hold
    params = I.Params(nx=64, ny=8, dx=1.0)
    with pytest.raises(swe.SweError) as e:
        swe.step_f32_noalloc(params, *([fake] * 8), (1 << 31) + 4, 0.0, 0.0)
    assert e.value.code == -1 and "INT_MAX" in str(e.value)
