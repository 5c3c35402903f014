"""Pins of the distributed sources of Eq. 1 (rainfall r, evaporation e,
infiltration i; m/s on every non-wall cell) in the FP64 oracle, against
closed forms on a flat frictionless closed basin: still water rises by
r tau per step (also from dry ground) and sinks by (e + i) tau until dry;
losses take water with its velocity (the velocity is unchanged), rain adds
water at rest (a flow slows to H U / (H + r tau)); and the volume of a
basin with terrain and gates changes by exactly r tau h^2 per non-gate cell
per step."""
import dataclasses

import numpy as np

import oracle
from paper_1705_00614_gb300 import inputs as I

TAU = 0.05


def _basin(n=24, H0=1.0, u0=0.0, **rates):
    p = I.Params(nx=n, ny=n, dx=2.0, dt_fixed=TAU, **rates)
    z = np.zeros((n, n))
    H = np.full((n, n), H0)
    return I.Problem("basin", p, z.copy(), z.copy(), H, H * u0, z.copy(), I.Sources.empty())


def _run(prob, nsteps):
    H, Qx, Qy, t, infos = oracle.run(prob, nsteps)
    return H, Qx, Qy, infos


def test_rain_on_still_water_and_on_dry_ground():
    r = 1.0e-3
    for H0 in (1.0, 0.0):
        H, Qx, Qy, _ = _run(_basin(H0=H0, rain_rate=r), 40)
        assert np.abs(H - (H0 + 40 * TAU * r)).max() <= 1e-12
        assert np.abs(Qx).max() == 0.0 and np.abs(Qy).max() == 0.0


def test_evaporation_and_infiltration_drain_still_water_until_dry():
    e, i = 2.0e-3, 3.0e-3
    H, Qx, Qy, _ = _run(_basin(H0=0.01, evap_rate=e, infil_rate=i), 30)
    # 0.01 m lasts 0.01 / 5e-3 = 2 s = 40 steps
    assert np.abs(H - (0.01 - 30 * TAU * (e + i))).max() <= 1e-12
    H, _, _, _ = _run(_basin(H0=0.01, evap_rate=e, infil_rate=i), 45)
    assert H.max() == 0.0


def test_losses_keep_the_velocity_and_rain_slows_the_flow():
    # one step of a uniform flow: cells 6 or more from the walls do not
    # feel them within a step
    u0, H0 = 0.5, 2.0
    c = (slice(8, 16), slice(8, 16))
    for rates, u_want in (({"evap_rate": 1e-3, "infil_rate": 2e-3}, u0),
                          ({"rain_rate": 4e-3}, H0 * u0 / (H0 + TAU * 4e-3))):
        H, Qx, _, _ = _run(_basin(H0=H0, u0=u0, **rates), 1)
        assert np.abs(Qx[c] / H[c] - u_want).max() <= 1e-13 * u0


def test_rain_volume_budget_over_terrain_with_gates():
    prob = I.with_gates(I.random_wet_dry(40, 36, seed=5, with_sources=False), seed=3, ngates=6)
    prob = dataclasses.replace(prob, params=dataclasses.replace(prob.params, dt_fixed=TAU, rain_rate=2e-3))
    h2 = prob.params.dx ** 2
    cells = prob.params.nx * prob.params.ny - int(prob.solid.sum())
    m0 = oracle.mass(prob, prob.H)
    H, Qx, Qy, infos = _run(prob, 10)
    src = sum(i["src_vol"] for i in infos)
    clip = sum(i["clip_vol"] for i in infos)
    assert abs(src - 10 * TAU * 2e-3 * cells * h2) <= 1e-9 * src
    assert abs(oracle.mass(prob, H) - m0 - src - clip) <= 1e-9 * m0
    # gate cells got no rain
    assert np.array_equal(H[prob.solid == 1], prob.H[prob.solid == 1])


def test_losses_beyond_the_depth_take_no_more_momentum_than_the_cell_holds():
    """Losses of (e + i) tau deeper than a moving layer, with rain that keeps
    the cell wet: the losses take the moving water (all of it) and its
    momentum, never more, so what is left is rain water at rest (zero
    momentum everywhere, not a reversed flow)."""
    H0, u0 = 0.001, 1.0
    prob = _basin(H0=H0, u0=u0, evap_rate=0.04, rain_rate=0.03)
    Hn, Qxn, Qyn, info, st = oracle.step(prob, prob.H, prob.Qx, prob.Qy, 0.0, stages=True)
    assert TAU * 0.04 > H0  # the losses exceed the layer
    assert np.all(st["ht"] > prob.params.eps)  # the rain keeps every cell wet
    assert np.abs(st["qtx"]).max() == 0.0 and np.abs(Qxn).max() == 0.0
    # away from the walls the (still moving) particles carry as much in as out
    assert np.abs(Hn[:, 3:-3] - (H0 + TAU * (0.03 - 0.04))).max() <= 1e-15
