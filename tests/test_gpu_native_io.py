"""Host arrays in the state's own precision (swe_set_state_native,
swe_get_state_native): the same state, checks and steps as the FP64 host
arrays of swe_set_state / swe_get_state."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec,dt", [("f32", np.float32), ("f64", np.float64)])
def test_native_state_round_trip_equals_fp64_path(swe, prec, dt):
    p = I.random_wet_dry(203, 131, seed=4)
    if prec == "f32":
        p = p.to_f32_values()
    with swe.Solver.from_problem(p, prec, seg_h=16) as a, swe.Solver.from_problem(p, prec, seg_h=16) as b:
        a.set_state(p.H, p.Qx, p.Qy, 1.5)
        b.set_state_native(p.H.astype(dt), p.Qx.astype(dt), p.Qy.astype(dt), 1.5)
        ia, ib = a.step(5), b.step(5)
        ga = a.get_state()
        out = [np.empty((p.params.ny, p.params.nx), dtype=dt) for _ in range(3)]
        tb = b.get_state_native_into(*out)
    assert ia == ib
    assert tb == ga[3]
    for x, y in zip(ga[:3], out):
        assert np.array_equal(np.asarray(x), y.astype(np.float64))


def test_native_upload_checks(swe):
    p = I.random_wet_dry(64, 40, seed=5).to_f32_values()
    with swe.Solver.from_problem(p, "f32") as s:
        H, Qx, Qy = (a.astype(np.float32) for a in (p.H, p.Qx, p.Qy))
        bad = H.copy()
        bad[3, 7] = -1e-3
        with pytest.raises(swe.SweError) as e:
            s.set_state_native(bad, Qx, Qy)
        assert e.value.code == -1
        nan = Qx.copy()
        nan[10, 2] = np.nan
        with pytest.raises(swe.SweError) as e:
            s.set_state_native(H, nan, Qy)
        assert e.value.code == -4
        # -0 is not a negative depth
        z = H.copy()
        z[0, 0] = -0.0
        s.set_state_native(z, Qx, Qy)
        with pytest.raises(ValueError):
            s.set_state_native(H.astype(np.float64), Qx, Qy)
