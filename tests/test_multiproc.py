"""The N > 1 path of bench.py on the CPU: two processes on the gloo backend
(the same calls as over NCCL, without a GPU).  Checked: the timed value is
the slowest rank's, work counts add up over ranks, the barrier releases
both ranks, and the ensemble's scenarios split across ranks disjointly and
completely, each rank building exactly the scenarios a single process
would."""
import json
import os
import socket

import numpy as np
import pytest

import bench
from paper_1705_00614_gb300 import inputs as I

WORLD = 2
ENS = dict(nmin=24, nmax=40, max_gates=3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.rank_barrier()
        mine = bench.shard(7, rank, world)
        shares = [None] * world
        dist.all_gather_object(shares, mine)
        idx = bench.shard(2 * world, rank, world)
        probs, gates = I.ensemble(2 * world, indices=idx, **ENS)
        cells = sum(p.params.nx * p.params.ny for p in probs)
        res = {
            "max": bench.over_ranks(1.5 + rank),
            "sum": bench.over_ranks(10 * (rank + 1), "sum"),
            "cells_job": bench.over_ranks(cells, "sum"),
            "shares": shares,
            "names": [p.name for p in probs],
            "bsum": [float(p.b.sum()) for p in probs],
            "gates": [g.ix.tolist() for g in gates],
        }
        bench.rank_barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    mp = pytest.importorskip("torch.multiprocessing")
    out = tmp_path_factory.mktemp("ranks")
    mp.start_processes(_worker, args=(WORLD, _free_port(), str(out)), nprocs=WORLD, join=True,
                       start_method="spawn")
    return [json.load(open(out / f"rank{r}.json")) for r in range(WORLD)]


def test_time_is_the_slowest_ranks_and_counts_add_up(results):
    for r in results:
        assert r["max"] == 1.5 + (WORLD - 1)
        assert r["sum"] == 10 * sum(range(1, WORLD + 1))


def test_units_split_disjointly_and_completely(results):
    shares = results[0]["shares"]
    assert shares == results[1]["shares"]
    flat = sorted(i for s in shares for i in s)
    assert flat == list(range(7))
    assert all(len(s) in (3, 4) for s in shares)


def test_each_rank_builds_the_single_process_scenarios(results):
    full, fgates = I.ensemble(2 * WORLD, **ENS)
    by_name = {p.name: (p, g) for p, g in zip(full, fgates)}
    seen = []
    for r in results:
        for name, bs, gx in zip(r["names"], r["bsum"], r["gates"]):
            p, g = by_name[name]
            assert bs == float(p.b.sum())
            assert gx == g.ix.tolist()
            seen.append(name)
    assert sorted(seen) == sorted(by_name)
    job = sum(p.params.nx * p.params.ny for p in full)
    assert all(r["cells_job"] == job for r in results)


def test_single_process_fallbacks():
    assert bench.over_ranks(3.25) == 3.25
    assert bench.over_ranks(3.25, "sum") == 3.25
    bench.rank_barrier()
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    with pytest.raises(ValueError):
        bench.shard(5, 2, 2)
    with pytest.raises(ValueError):
        I.ensemble(3, indices=[3], **ENS)
    # whole-job rate: units of all ranks over the slowest rank's time
    assert bench.job_rate(2e9, 500.0) == pytest.approx(4.0)
    assert np.isclose(bench.job_rate(WORLD * 1e9, 1000.0), WORLD)
