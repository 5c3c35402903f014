"""The default benchmark line's secondary entries (CPU only): which fields of
a secondary workload's line are kept, that each workload runs with its own
steps on a copy of the arguments, and that a failing workload is reported
as an error entry instead of ending the run."""
import argparse
import types

import bench


class _FakeCuda:
    def __init__(self):
        self.streams = 0

    def Stream(self):
        self.streams += 1
        return types.SimpleNamespace(cuda_stream=self.streams)

    def set_stream(self, s):
        self.current = s

    def synchronize(self):
        pass


def _line(workload, value):
    return {"metric": "m", "value": value, "unit": "u", "n_gpus": 1, "steps": 7, "warmup": 3, "ms_per_step": 1.5,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "cells": 10, "scenarios": 2, "parallelism": "single GPU"},
            "roofline": {"bound": "hbm", "frac": 0.1}, "gpu_launches": 7, "clocks": {"sm_mhz": 1.0},
            "cpu_baseline": None, "e2e": None}


def test_entry_keeps_the_measurement_and_drops_the_rest():
    e = bench.secondary_entry(_line("ensemble-64", 3.0))
    assert e["workload"] == "ensemble-64" and e["value"] == 3.0 and e["ms_per_step"] == 1.5
    assert e["roofline"] == {"bound": "hbm", "frac": 0.1} and e["clocks"] == {"sm_mhz": 1.0}
    assert e["config"] == {"cells": 10, "scenarios": 2}
    assert "cpu_baseline" not in e and "e2e" not in e and "data" not in e


def test_each_workload_runs_on_a_copy_and_errors_are_reported(monkeypatch):
    seen = []

    def ok(a, torch, swe, stream, rank, world, emit=True):
        assert emit is False and rank == 0 and world == 1
        seen.append((a.workload, a.steps, a.warmup))
        return _line(a.workload, 5.0)

    def boom(a, torch, swe, stream, rank, world, emit=True):
        seen.append((a.workload, a.steps, a.warmup))
        raise RuntimeError("device wait timed out")

    monkeypatch.setattr(bench, "_fake_ok", ok, raising=False)
    monkeypatch.setattr(bench, "_fake_boom", boom, raising=False)
    monkeypatch.setattr(bench, "SECONDARY", (("ensemble-4", 11, 3, "_fake_boom"), ("cnn-64sq", 13, 4, "_fake_ok")))
    args = argparse.Namespace(workload="floodplain", steps=200, warmup=5, precision="f32")
    torch = types.SimpleNamespace(cuda=_FakeCuda())
    out = bench.run_secondary(args, torch, None)
    assert seen == [("ensemble-4", 11, 3), ("cnn-64sq", 13, 4)]
    assert out[0] == {"workload": "ensemble-4", "error": "RuntimeError: device wait timed out"}
    assert out[1]["workload"] == "cnn-64sq" and out[1]["value"] == 5.0
    assert (args.workload, args.steps, args.warmup) == ("floodplain", 200, 5)
    assert torch.cuda.streams == 2


def test_default_secondary_workloads_exist():
    for wl, steps, warmup, fn in bench.SECONDARY:
        assert callable(getattr(bench, fn))
        assert steps > 0 and warmup >= 3
        assert wl.split("-")[0] in ("ensemble", "cnn")


def test_only_the_default_one_gpu_line_gets_secondary_runs():
    base = dict(workload="floodplain-16384sq-dx2m-flooded", precision="f32", mode="fused", skip_dry=False,
                no_secondary=False)
    default = base["workload"]

    def wants(world=1, **kw):
        return bench.wants_secondary(argparse.Namespace(**{**base, **kw}), world, default)

    assert wants()
    assert not wants(world=2)
    assert not wants(no_secondary=True)
    assert not wants(workload="floodplain-4096sq-dx5m-flooded")
    assert not wants(precision="f64")
    assert not wants(mode="staged")
    assert not wants(skip_dry=True)
