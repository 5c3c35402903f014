"""The oracle arm of bench.py (`--impl reference`) on the CPU: one JSON line
with the same metric and unit as the GPU arm, the oracle's rate as value,
cpu_baseline and e2e alike, no host-device bytes; fewer than 3 warm-up steps
are refused."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--workload", "floodplain-2048sq-dx10m-flooded", "--ref-crop", "64",
        "--cpu-procs", "2", "--steps", "2"]


def _run(*extra):
    return subprocess.run([sys.executable, "bench.py", *ARGS, *extra], cwd=ROOT, capture_output=True, text=True,
                          timeout=300)


def test_reference_line():
    r = _run("--warmup", "3")
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "floodplain-2048sq-dx10m-flooded"


def test_short_warmup_refused():
    r = _run("--warmup", "2")
    assert r.returncode != 0
    assert "--warmup must be >= 3" in r.stderr
