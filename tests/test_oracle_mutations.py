"""The oracle's pins catch plausible mistakes.

Each case plants one slip in a copy of the oracle source (a flipped sign, a
wrong factor, a swapped index, a dropped term), builds it with gcc on the
CPU, and checks that at least one pin of test_oracle_pins.py or
test_oracle_rain.py fails against
the mutated build.  Mistakes are planted only in the oracle, never in the
CUDA path.
"""
import os
import tempfile

import pytest

import oracle
from tests import test_oracle_pins as P
from tests import test_cnn_oracle_pins as CP
from tests import test_oracle_rain as R

_SRC = os.path.join(os.path.dirname(oracle.__file__), "swe_oracle.c")

# (name, exact source text, replacement, pins to try)
MUTANTS = [
    ("pressure sign", "double coef = -g / (4.0 * h * hs[k]);", "double coef = g / (4.0 * h * hs[k]);",
     ["test_stoker_dam_break_256"]),
    ("pressure factor", "double coef = -g / (4.0 * h * hs[k]);", "double coef = -g / (2.0 * h * hs[k]);",
     ["test_stoker_dam_break_256"]),
    ("reconstruction uses own bed", "double bs = dmax(bL, bR);\n    double hl", "double bs = bL;\n    double hl",
     ["test_lake_at_rest_fractal_islands"]),
    ("Coriolis sign", "double aCx = p->f * uy[k], aCy = -p->f * ux[k];",
     "double aCx = -p->f * uy[k], aCy = p->f * ux[k];", ["test_coriolis_inertial_rotation_second_order"]),
    ("wind without depth", "double cw = p->ca * p->ra * wm / hs[k];", "double cw = p->ca * p->ra * wm;",
     ["test_wind_spin_up_second_order"]),
    ("friction exponent", "um / (hs[k] * cbrt(hs[k]));", "um / cbrt(hs[k]);",
     ["test_friction_decay_matches_manning_ode"]),
    ("viscosity north neighbour index", "dvx = (j < ny - 1 && wet[k + nx]) ? ux[k + nx] - ux[k] : 0.0;",
     "dvx = (j < ny - 1 && wet[k + nx]) ? ux[k + 1] - ux[k] : 0.0;", ["test_viscous_shear_mode_decay"]),
    ("viscosity dropped h^2", "double cv = p->nu / (h * h);", "double cv = p->nu / h;",
     ["test_viscous_shear_mode_decay"]),
    ("full-step predictor", "const double th = 0.5 * tau;", "const double th = tau;",
     ["test_coriolis_inertial_rotation_second_order"]),
    ("corrector from U*", "utx[k] = wet[k] ? (ux[k] + tau * ax2[k])", "utx[k] = wet[k] ? (usx[k] + tau * ax2[k])",
     ["test_coriolis_inertial_rotation_second_order"]),
    ("momentum upwind swapped", "FQx = FH * (FH >= 0.0 ? wl[3] : wr[3]);", "FQx = FH * (FH >= 0.0 ? wr[3] : wl[3]);",
     ["test_stoker_dam_break_256"]),
    ("final update sign", "double fh = (fxl[fw] - fxl[fe])", "double fh = (fxl[fe] - fxl[fw])",
     ["test_stoker_dam_break_256"]),
    ("y faces read x fluxes", "double fqy = (fxl[2 * NFX + fw] - fxl[2 * NFX + fe]) + (fyl[2 * NFY + fs] - fyl[2 * NFY + fn]);",
     "double fqy = (fxl[2 * NFX + fw] - fxl[2 * NFX + fe]) + (fyl[NFY + fs] - fyl[NFY + fn]);",
     ["test_transpose_symmetry_random_wet_dry"]),
    ("minmod picks the larger slope", "if (a > 0.0 && b > 0.0) return a < b ? a : b;",
     "if (a > 0.0 && b > 0.0) return a > b ? a : b;", ["test_tvd_transverse_velocity_advection"]),
    ("star sound speed sign", "double cs = 0.5 * (cl + cr) + 0.25 * (ul - ur);",
     "double cs = 0.5 * (cl + cr) + 0.25 * (ur - ul);", ["test_riemann_two_rarefactions_is_exact"]),
    ("dry-bed fan speed", "if (ul - cl >= 0.0) { h = hl; u = ul; }\n        else if (ul + 2.0 * cl > 0.0) { double c = (ul + 2.0 * cl) / 3.0; h = c * c / g; u = c; }\n    } else if (dl)",
     "if (ul - cl >= 0.0) { h = hl; u = ul; }\n        else if (ul + 2.0 * cl > 0.0) { double c = (ul + cl) / 3.0; h = c * c / g; u = c; }\n    } else if (dl)",
     ["test_riemann_dry_bed_fan_and_mirror"]),
    ("Courant number ignored", "tau = dmin(p->dt_max, p->cfl * p->dx / smax);", "tau = dmin(p->dt_max, p->dx / smax);",
     ["test_stoker_dam_break_256"]),
    ("source at t_n", "sig[k] = source_rate(src, m, t + th);", "sig[k] = source_rate(src, m, t);",
     ["test_source_volume_matches_hydrograph_integral"]),
    ("drain volume unclamped", "ht[k] = dmax(0.0, hp);", "ht[k] = hp;",
     ["test_drain_on_dry_ground_removes_nothing"]),
    ("evaporation adds water", "ht[k] = dmax(0.0, hp + tau * (p->rain - loss));",
     "ht[k] = dmax(0.0, hp + tau * (p->rain + loss));",
     ["test_evaporation_and_infiltration_drain_still_water_until_dry"]),
    ("losses leave the momentum", "qtx[k] = qtx[k] - taken * utx[k];", "qtx[k] = qtx[k];",
     ["test_losses_keep_the_velocity_and_rain_slows_the_flow"]),
    ("rain on gates", "if (!solid[k] && (p->rain != 0.0", "if ((p->rain != 0.0",
     ["test_rain_volume_budget_over_terrain_with_gates"]),
    ("drain keeps the momentum of a negative depth", "if (sig[k] > 0.0 || hp > 0.0) {", "if (1) {",
     ["test_drain_emptying_a_moving_cell_leaves_no_momentum"]),
    ("losses take more than the cell holds", "double taken = dmin(tau * loss, dmax(0.0, hp));",
     "double taken = tau * loss;",
     ["test_losses_beyond_the_depth_take_no_more_momentum_than_the_cell_holds"]),
    ("particle speed dropped", "double s = dmax(us, dmax(upx, upy));", "double s = us;",
     ["test_time_step_from_particle_speed"]),
    ("particle speed without h", "double upx = fabs(ux[k] + sgn(ax[k]) * sqrt(p->dx * fabs(ax[k])));",
     "double upx = fabs(ux[k] + sgn(ax[k]) * sqrt(fabs(ax[k])));", ["test_time_step_from_particle_speed"]),
    ("particle speed without sign", "double upx = fabs(ux[k] + sgn(ax[k]) * sqrt(p->dx * fabs(ax[k])));",
     "double upx = fabs(ux[k] + sqrt(p->dx * fabs(ax[k])));", ["test_time_step_from_particle_speed"]),
    ("particle speed y from a_x", "double upy = fabs(uy[k] + sgn(ay[k]) * sqrt(p->dx * fabs(ay[k])));",
     "double upy = fabs(uy[k] + sgn(ax[k]) * sqrt(p->dx * fabs(ax[k])));", ["test_time_step_from_particle_speed"]),
    ("wave speed from the sum of components", "double us = dmax(fabs(ux[k]), fabs(uy[k])) + c;",
     "double us = fabs(ux[k]) + fabs(uy[k]) + c;", ["test_time_step_from_wave_speed_two_components"]),
    ("closure correction of Q_x applied to Q_y", "fqy = fqy + bounded(corr[2 * N + k], fqy, corr_bound);",
     "fqy = fqy + bounded(corr[N + k], fqy, corr_bound);",
     ["test_oracle_step_applies_flux_corrections_in_the_final_update"]),
    ("closure correction subtracted", "fh = fh + bounded(corr[k], fh, corr_bound);",
     "fh = fh - bounded(corr[k], fh, corr_bound);",
     ["test_oracle_step_applies_flux_corrections_in_the_final_update"]),
    ("bound without the magnitude", "double lim = beta * fabs(f);", "double lim = beta * f;",
     ["test_bounded_corrections_are_clamped_to_a_fraction_of_the_flux_sums"]),
    ("momentum correction bounded by the mass flux", "fqx = fqx + bounded(corr[N + k], fqx, corr_bound);",
     "fqx = fqx + bounded(corr[N + k], fh, corr_bound);",
     ["test_bounded_corrections_are_clamped_to_a_fraction_of_the_flux_sums"]),
]


def _cases(fn):
    """Argument tuples of a pin: its parametrize cases, or one empty call."""
    marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
    if not marks:
        return [()]
    names, values = marks[0].args[0], marks[0].args[1]
    single = "," not in names if isinstance(names, str) else len(names) == 1
    return [(v,) if single else tuple(v) for v in values]


@pytest.fixture(scope="module")
def tmpdir_mod():
    with tempfile.TemporaryDirectory() as d:
        yield d


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, pins, tmpdir_mod, monkeypatch):
    src = open(_SRC).read()
    assert src.count(old) == 1, f"mutation site for '{name}' not found exactly once"
    path = os.path.join(tmpdir_mod, name.replace(" ", "_") + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = oracle.build(force=True, src=path, out=path[:-2] + ".so")
    monkeypatch.setattr(oracle, "_lib", oracle.lib(so))
    caught = []
    for pin in pins:
        fn = getattr(P, pin, None) or getattr(R, pin, None) or getattr(CP, pin)
        try:
            for args in _cases(fn):
                fn(*args)
        except (AssertionError, RuntimeError, FloatingPointError, ValueError, ZeroDivisionError):
            caught.append(pin)
            break
    assert caught, f"no pin caught the planted mistake '{name}'"
