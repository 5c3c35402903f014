"""The closure benchmark's choice of correction scale on the validation
seeds (CPU only): the largest scale within the error bar, NaN never passes,
the smallest error when none passes, the first listed among equal scales."""
import math

import bench

NAMES = ["closed_a1", "closed_a0.5", "closed_a0.25", "closed_a0.1"]
ALPHAS = [1.0, 0.5, 0.25, 0.1]


def test_largest_scale_within_the_bar():
    err = {"closed_a1": 0.012, "closed_a0.5": 0.009, "closed_a0.25": 0.004, "closed_a0.1": 0.003}
    assert bench.choose_on_validation(NAMES, ALPHAS, err) == "closed_a0.5"


def test_a_diverged_run_never_passes():
    err = {"closed_a1": math.nan, "closed_a0.5": 0.02, "closed_a0.25": 0.008, "closed_a0.1": 0.003}
    assert bench.choose_on_validation(NAMES, ALPHAS, err) == "closed_a0.25"


def test_smallest_error_when_none_passes():
    err = {"closed_a1": math.nan, "closed_a0.5": 0.05, "closed_a0.25": 0.03, "closed_a0.1": 0.04}
    assert bench.choose_on_validation(NAMES, ALPHAS, err) == "closed_a0.25"


def test_equal_scales_keep_the_first_listed():
    names = ["closed_a1", "closed_a1_momentum_only", "closed_a0.5"]
    err = {"closed_a1": 0.005, "closed_a1_momentum_only": 0.004, "closed_a0.5": 0.001}
    assert bench.choose_on_validation(names, [1.0, 1.0, 0.5], err) == "closed_a1"


def test_the_bar_is_inclusive():
    err = {"closed_a1": 0.01, "closed_a0.5": 0.0, "closed_a0.25": 0.0, "closed_a0.1": 0.0}
    assert bench.choose_on_validation(NAMES, ALPHAS, err) == "closed_a1"
