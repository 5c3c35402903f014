"""Two-level nesting through the C ABI (swe_nest_*): a fine patch with a
ghost ring, 4 sub-steps per coarse step, ghosts from the coarse grid and
4 x 4 feedback.  FP64 against the nesting oracle (oracle/nest_oracle.py),
FP32 on FP32-rounded inputs, still water, and what the patch buys over the
coarse grid alone against a fine solution of the whole domain."""
import dataclasses
import os
import sys

import numpy as np
import pytest

from oracle import nest_oracle as N
from paper_1705_00614_gb300 import inputs as I

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from test_nest_oracle import _nest_setup  # noqa: E402

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


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _rounded(coarse, fine, b_ext, n_ext):
    return coarse.to_f32_values(), fine.to_f32_values(), _f32(b_ext), _f32(n_ext)


def _run_gpu(swe, prec, coarse, fine, b_ext, n_ext, ix0, iy0, ncoarse):
    with swe.Solver.from_problem(coarse, prec) as c, swe.Solver.from_problem(fine, prec, ghost_ring=True) as f:
        f.set_terrain_ext(b_ext, n_ext)
        f.set_state(fine.H, fine.Qx, fine.Qy, 0.0)
        with swe.Nest(c, f, ix0, iy0) as nest:
            ic, jf = nest.step(ncoarse)
        return c.get_state(), f.get_state(), ic, jf


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-4)])
def test_nest_matches_oracle(swe, prec, tol):
    coarse, fine, b_ext, n_ext, ix0, iy0 = _nest_setup(31)
    if prec == "f32":
        coarse, fine, b_ext, n_ext = _rounded(coarse, fine, b_ext, n_ext)
    cg, fg, ic, jf = _run_gpu(swe, prec, coarse, fine, b_ext, n_ext, ix0, iy0, 3)
    co, fo = N.nest_run(coarse, fine, b_ext, n_ext, ix0, iy0, 3)
    for q in range(3):
        assert _rel(cg[q], co[q]) <= tol, ("coarse", q, _rel(cg[q], co[q]))
        assert _rel(fg[q], fo[q]) <= tol, ("fine", q, _rel(fg[q], fo[q]))
    # each step's tau is rounded to the state precision (0.2 in FP32 is 0.2 + 3e-9)
    ttol = 1e-12 if prec == "f64" else 1e-7
    assert abs(ic["t"] - 0.6) <= ttol and abs(jf["t"] - 0.6) <= ttol
    assert ic["step"] == 3 and jf["step"] == 12


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_nested_still_water_stays_still(swe, prec, tol):
    coarse, fine, b_ext, n_ext, ix0, iy0 = _nest_setup(12, still=True)
    if prec == "f32":
        coarse, fine, b_ext, n_ext = _rounded(coarse, fine, b_ext, n_ext)
    cg, fg, _, _ = _run_gpu(swe, prec, coarse, fine, b_ext, n_ext, ix0, iy0, 5)
    assert np.abs(fg[0] - fine.H).max() <= tol * max(1.0, fine.H.max())
    assert np.abs(cg[0] - coarse.H).max() <= tol * max(1.0, coarse.H.max())
    for a in (fg[1], fg[2], cg[1], cg[2]):
        assert np.abs(a).max() <= tol


def test_patch_is_closer_to_the_fine_solution_than_the_coarse_grid(swe):
    """A flood release crossing the patch: on the patch, the nested fine
    solution is closer to a fine solution of the whole domain than the
    coarse grid alone (refined piecewise constant)."""
    nxc, nyc, ix0, iy0, wc, hc = 40, 24, 14, 6, 12, 12
    base = I.floodplain(4 * nxc, 5.0, 4242, 4243, ny=4 * nyc, nsrc=1)
    from paper_1705_00614_gb300 import closure as CL
    base = CL.dam_release(dataclasses.replace(base, sources=I.Sources.empty()), quantile=0.5, rise=1.5, frac=0.3)
    bf = base.b
    Hf0, Qxf0, Qyf0 = base.H, base.Qx, base.Qy

    def r4(a):
        return a.reshape(nyc, 4, nxc, 4).mean(axis=(1, 3))

    pc = dataclasses.replace(base.params, nx=nxc, ny=nyc, dx=20.0, dt_fixed=0.2)
    coarse = I.Problem("coarse", pc, r4(bf), r4(base.n_manning), r4(Hf0), r4(Qxf0), r4(Qyf0), I.Sources.empty())
    x0, y0, nx, ny = 4 * ix0, 4 * iy0, 4 * wc, 4 * hc
    sl = (slice(y0, y0 + ny), slice(x0, x0 + nx))
    esl = (slice(y0 - N.PAD, y0 + ny + N.PAD), slice(x0 - N.PAD, x0 + nx + N.PAD))
    pf = dataclasses.replace(base.params, nx=nx, ny=ny, dt_fixed=0.05)
    fine = I.Problem("fine", pf, bf[sl], base.n_manning[sl], Hf0[sl], Qxf0[sl], Qyf0[sl], I.Sources.empty())
    full = dataclasses.replace(base, params=dataclasses.replace(base.params, dt_fixed=0.05))
    ncoarse = 60
    cg, fg, _, _ = _run_gpu(swe, "f32", coarse.to_f32_values(), fine.to_f32_values(), _f32(bf[esl]),
                            _f32(base.n_manning[esl]), ix0, iy0, ncoarse)
    with swe.Solver.from_problem(full.to_f32_values(), "f32") as s:
        s.step(4 * ncoarse)
        Href = s.get_state()[0][sl]
    with swe.Solver.from_problem(coarse.to_f32_values(), "f32") as s:
        s.step(ncoarse)
        Hc = np.kron(s.get_state()[0], np.ones((4, 4)))[sl]
    # compare free surfaces where the reference is wet
    wet = Href > 1e-3
    e_nest = np.linalg.norm((fg[0] - Href)[wet]) / np.linalg.norm(Href[wet])
    e_coarse = np.linalg.norm((Hc - Href)[wet]) / np.linalg.norm(Href[wet])
    print("patch vs fine reference: nested", e_nest, "coarse only", e_coarse)
    assert e_nest < e_coarse
