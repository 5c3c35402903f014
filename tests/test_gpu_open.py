"""Open (outflow) boundaries through the C ABI (ghost_ring = 2): the ring
takes the nearest interior cell's state before every step.  FP64 against
the oracle's construction (oracle/nest_oracle.open_run) and uniform flow
leaving the grid unchanged, FP64 and FP32."""
import os
import sys

import numpy as np
import pytest

from oracle import nest_oracle as N
from paper_1705_00614_gb300 import inputs as I

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from test_nest_oracle import _open_basin  # noqa: E402

pytestmark = pytest.mark.gpu
P = N.PAD


@pytest.fixture(scope="module")
def swe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1705_00614_gb300 import build, swe as S
    build.build()
    S.load()
    return S


def _run(swe, prob, b_ext, prec, nsteps):
    with swe.Solver.from_problem(prob, prec, ghost_ring=2) as s:
        s.set_terrain_ext(b_ext)
        s.set_state(prob.H, prob.Qx, prob.Qy, 0.0)
        s.step(nsteps)
        return s.get_state()


@pytest.mark.parametrize("prec,tol,dt", [("f64", 1e-12, 0.05), ("f32", 1e-5, 0.05), ("f64", 1e-12, 0.0)])
def test_open_boundary_matches_oracle(swe, prec, tol, dt):
    """A dam break over terrain leaving through the east and south edges;
    with dt = 0 the steps follow the CFL condition over the filled ring as
    well (the oracle steps the padded extent as one grid)."""
    base = I.random_wet_dry(60, 44, seed=17, with_sources=False)
    import dataclasses
    p = dataclasses.replace(base.params, dt_fixed=dt)
    ny, nx = base.H.shape
    H = base.H + np.where(np.arange(nx) < 20, 1.0, 0.0)[None, :]
    b_ext = np.pad(base.b, P, mode="edge")
    b_ext[:P, :] = 1e30
    b_ext[:, :P] = 1e30
    prob = dataclasses.replace(base, params=p, H=H)
    if prec == "f32":
        prob = prob.to_f32_values()
        b_ext = np.asarray(b_ext, np.float32).astype(np.float64)
    g = _run(swe, prob, b_ext, prec, 6)
    o = N.open_run(prob, b_ext, None, 6)
    for a, b in zip(g[:3], o):
        assert np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1.0)
    if dt == 0.0:
        assert abs(g[3] - N.open_run_time(prob, b_ext, None, 6)) <= 1e-13 * g[3]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_uniform_flow_leaves_unchanged(swe, prec, tol):
    prob, b_ext = _open_basin()
    if prec == "f32":
        prob = prob.to_f32_values()
    H, Qx, Qy, _ = _run(swe, prob, b_ext, prec, 40)
    assert np.abs(H - prob.H).max() <= tol * 2.0
    assert np.abs(Qx - prob.Qx).max() <= tol * 2.0 and np.abs(Qy - prob.Qy).max() <= tol * 2.0


def test_batch_rejects_ghost_ring_contexts(swe):
    """A batched step runs no ghost fills, so ghost-ring contexts are refused."""
    prob, b_ext = _open_basin(n=24)
    with swe.Solver.from_problem(prob, "f64", ghost_ring=2) as s:
        s.set_terrain_ext(b_ext)
        s.set_state(prob.H, prob.Qx, prob.Qy, 0.0)
        with pytest.raises(swe.SweError) as e:
            swe.Batch([s])
        assert e.value.code == -1
