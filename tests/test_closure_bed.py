"""The coarse grid the closure works on (closure.coarse_problem): with the
volume-matched bed, still fine water gives a coarse free surface that is
flat wherever a block holds water, the coarse volume is the fine volume
exactly, fully wet and fully dry blocks keep the 4 x 4 mean bed, and the
coarse lake stays at rest under the FP64 oracle (with the mean bed the
partly wet cells stand above the lake and the water moves)."""
import dataclasses

import numpy as np

import oracle
from paper_1705_00614_gb300 import closure as CL
from paper_1705_00614_gb300 import inputs as I


def _still(n=64, seed=3):
    p = I.lake_at_rest(n, 5.0, seed, eta0=12.0, nu=0.0, coriolis_f=0.0)
    return dataclasses.replace(p, params=dataclasses.replace(p.params, wind_x=0.0, wind_y=0.0))


def test_volume_bed_flat_surface_and_exact_volume():
    fine = _still()
    cm = CL.coarse_problem(fine, "mean")
    cv = CL.coarse_problem(fine, "volume")
    assert np.array_equal(cv.H, cm.H)  # depth is the 4 x 4 mean either way
    assert cv.H.sum() * 16 == fine.H.sum()
    wet = cv.H > 0
    eta = (cv.H + cv.b)[wet]
    assert np.abs(eta - 12.0).max() <= 1e-12
    blocks = (fine.H > 0).reshape(16, 4, 16, 4)
    full = blocks.all(axis=(1, 3)) | ~blocks.any(axis=(1, 3))
    assert np.array_equal(cv.b[full], cm.b[full])
    # the mean bed leaves partly wet cells standing above the lake
    assert np.abs((cm.H + cm.b)[wet] - 12.0).max() > 1e-3


def test_volume_bed_coarse_lake_stays_at_rest():
    fine = _still()
    for bed, still in (("volume", True), ("mean", False)):
        c = CL.with_dt(CL.coarse_problem(fine, bed), 0.5)
        H, Qx, Qy, _, _ = oracle.run(c, 20)
        moved = max(np.abs(Qx).max(), np.abs(Qy).max())
        assert (moved <= 1e-12) == still, (bed, moved)
