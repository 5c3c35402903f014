"""Failure paths on the GPU without a fault or a hang: a bounded device wait
on an mbarrier phase that nothing completes (the wait the step kernels use
for their input rows) runs out, sets the timeout bit, comes back as
SWE_ERR_DEVICE_TIMEOUT, and the device keeps working."""
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


def test_bounded_wait_runs_out_and_the_device_stays_usable(swe):
    for limit in (5, 50):
        with pytest.raises(swe.SweError) as e:
            swe.check_bounded_wait(limit)
        assert e.value.code == -6
    p = I.dam_break(64, 1.0, ny=8)
    H, Qx, Qy, t, _ = oracle.run(p, 3)
    with swe.Solver.from_problem(p, "f64") as s:
        s.step(3)
        g = s.get_state()
    assert np.abs(g[0] - H).max() <= 1e-12 * np.abs(H).max()
