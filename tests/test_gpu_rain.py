"""Rain, evaporation and infiltration (distributed sources of Eq. 1) through
the C ABI: staged and fused FP64 against the oracle (1e-12 per step, with
gates and the CFL time step), fused FP32 (1e-5), the closed form of rain on
still water, and dry-tile skipping switched off while it rains."""
import dataclasses

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


def _problem(prec, rates):
    p = I.with_gates(I.random_wet_dry(150, 130, seed=71), seed=2, ngates=5)
    p = dataclasses.replace(p, params=dataclasses.replace(p.params, **rates))
    return p.to_f32_values() if prec == "f32" else p


RATES = [{"rain_rate": 3e-3}, {"evap_rate": 2e-3, "infil_rate": 4e-3},
         {"rain_rate": 1e-3, "evap_rate": 5e-4, "infil_rate": 5e-4}]


@pytest.mark.parametrize("rates", RATES, ids=["rain", "losses", "both"])
@pytest.mark.parametrize("mode", ["staged", "fused"])
def test_f64_matches_oracle(swe, mode, rates):
    p = _problem("f64", rates)
    with swe.Solver.from_problem(p, "f64", mode=mode) as s:
        H, Qx, Qy, t = p.H, p.Qx, p.Qy, 0.0
        for _ in range(3):
            H, Qx, Qy, info, _ = oracle.step(p, H, Qx, Qy, t)
            t = info["t_new"]
            rep = s.step(1)
            g = s.get_state()
            assert abs(g[3] - t) <= 1e-13 * t
            for a, o in zip(g[:3], (H, Qx, Qy)):
                assert np.abs(a - o).max() <= 1e-12 * max(np.abs(o).max(), 1e-6)
            assert abs(rep["src_vol"] - info["src_vol"]) <= 1e-10 * max(abs(info["src_vol"]), 1.0)


@pytest.mark.parametrize("rates", RATES, ids=["rain", "losses", "both"])
def test_f32_fused_matches_oracle(swe, rates):
    p = _problem("f32", rates)
    H, Qx, Qy, info, _ = oracle.step(p, p.H, p.Qx, p.Qy, 0.0)
    with swe.Solver.from_problem(p, "f32") as s:
        s.step(1)
        g = s.get_state()
    for a, o in zip(g[:3], (H, Qx, Qy)):
        assert np.abs(a - o).max() <= 1e-5 * max(np.abs(o).max(), 1e-3)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_rain_on_still_water(swe, prec, tol):
    n, tau, r, H0 = 64, 0.05, 2e-3, 1.5
    par = I.Params(nx=n, ny=n, dx=2.0, dt_fixed=tau, rain_rate=r)
    z = np.zeros((n, n))
    p = I.Problem("basin", par, z, z.copy(), np.full((n, n), H0), z.copy(), z.copy(), I.Sources.empty())
    with swe.Solver.from_problem(p, prec) as s:
        info = s.step(50)
        H, Qx, Qy, _ = s.get_state()
    assert np.abs(H - (H0 + 50 * tau * r)).max() <= tol * H0
    assert np.abs(Qx).max() <= tol and np.abs(Qy).max() <= tol
    # the reported volume is the sum of H~ - H: in FP32 each 1e-4 m increment
    # on a 1.5 m depth carries the depth's rounding (1.2e-7 m)
    want = tau * r * n * n * 4.0
    assert abs(info["src_vol"] - want) <= (1e-9 if prec == "f64" else 2e-3) * want


def test_rain_switches_skipping_off(swe):
    p = _problem("f32", {"rain_rate": 3e-3})
    with swe.Solver.from_problem(p, "f32", seg_h=32, skip_dry=True) as a, \
            swe.Solver.from_problem(p, "f32", seg_h=32) as b:
        ra, rb = a.step(5), b.step(5)
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    assert ra["skipped"] == 0 and ra["mass"] == rb["mass"]
