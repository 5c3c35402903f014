"""Benchmark of the CSPH-TVD time step on one GB300 (or N replicas).

Default workload: the 16384^2 fractal floodplain at dx = 2 m (268M cells,
FP32, every physics term of Eqs. 1-4 on, 100-cell inflow strip), flooded to
the median terrain height so about half of the cells are wet (the paper's
emergency-discharge run had 35-60% water, Sec. 5).  A step is one pass of
the whole hot path: forces, CFL time step, Lagrangian predictor-corrector,
Eulerian fluxes and final update, all in the fused kernel (one launch).

Prints one JSON line:
  value        cell-updates/s (Gcell/s) of K device-resident steps (one CUDA
               graph of K launches), max over ranks, all ranks' cells counted
  e2e          the same metric through the C ABI with host buffers: each
               step uploads the state from pinned host memory in the state's
               precision (swe_set_state_native), advances one step
               (swe_step) and reads the state back (swe_get_state_native),
               copies inside the timed region; fp64_host: the same with the
               FP64 host arrays of swe_set_state / swe_get_state
  roofline     the fused kernel against measured HBM copy bandwidth:
               32 algorithmic bytes per cell (read H, Qx, Qy, b, n; write
               H, Qx, Qy in FP32) over its CUDA-event time per launch;
               traffic = DRAM bytes per launch from the committed ncu
               summary (the kernel also stores the state's accelerations,
               48 B/cell in all)
  alu_roofline the same kernel against the instruction-issue ceiling it is
               actually bound by: warp instructions per cell (committed ncu
               summary) x cells / time, over SMs x 4 schedulers x the SM
               clock sampled during the timed region
  cpu_baseline the FP64 CPU oracle on a bounded crop of the same workload,
               one process per host core
  secondary    (one GPU, default workload, unless --no-secondary) short runs
               of the other measured paths, after the timed region above and
               each in its own: the batched ensemble (64 scenarios of
               512^2-2048^2, 500 steps with gate toggles; the HBM roofline of
               k_fused_batch) and the closure network's training step on a
               2048^2 grid (the BF16 tensor roofline); a path that fails
               reports its error instead of a value
``--impl reference`` times the oracle alone on the host cores (the same way).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1705_00614_gb300 import inputs as I  # noqa: E402

METRIC = "Gcell-updates/s and HBM-roofline %; CNN-closure vs fine solve at ≤1% L2"
UNIT = "Gcell-updates/s"
BYTES_PER_CELL = {"f32": 32, "f64": 64}
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy bandwidth is the roofline peak)
KERNEL_SOURCES = ["paper_1705_00614_gb300/csrc/swe_kernels.cuh", "paper_1705_00614_gb300/csrc/swe_math.cuh",
                  "paper_1705_00614_gb300/csrc/swe_launch.h"]


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def over_ranks(x, op="max"):
    """x combined over the ranks of the initialised process group ("max" or
    "sum"; a float64 all-reduce on the backend's device); x itself in a
    single-process run.  Timing takes the slowest rank, counts of work the
    sum: nothing of the solver's data crosses ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def rank_barrier():
    """Barrier across the ranks of the initialised process group (no-op in a
    single-process run)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def shard(n, rank, world):
    """Indices of the n independent units (ensemble scenarios) that `rank`
    of `world` runs: round robin, disjoint across ranks, together all n."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world {world}")
    return list(range(rank, n, world))


def job_rate(units, ms):
    """Whole-job throughput in G-units/s: units processed by all ranks over
    the slowest rank's time (ms)."""
    return units / (ms * 1e-3) / 1e9


def flooded_workload(name):
    """The benchmark problem: a named floodplain, filled to its median
    terrain height (still water), keeping the inflow strip and physics.
    Without the "-flooded" suffix the floodplain starts dry (the inflow
    strip is the only water), the case dry-tile skipping is for."""
    base = name.replace("-flooded", "")
    p = I.workload(base)
    if not name.endswith("-flooded"):
        return p.to_f32_values(), None
    eta0 = float(np.median(p.b))
    H = np.maximum(0.0, eta0 - p.b)
    z = np.zeros_like(H)
    return I.Problem(name, p.params, p.b, p.n_manning, H, z, z.copy(), p.sources).to_f32_values(), eta0


def flooded_ensemble(n, rank=0, world=1):
    """The batched-ensemble workload of one rank: its share (round robin) of
    an ensemble of n x world scenarios with N uniform in [512, 2048], each
    filled to its median terrain height.  One rank runs all n."""
    probs, gates = I.ensemble(n * world, indices=shard(n * world, rank, world))
    out = []
    for p in probs:
        eta0 = float(np.median(p.b))
        H = np.maximum(0.0, eta0 - p.b)
        z = np.zeros_like(H)
        out.append(I.Problem(p.name, p.params, p.b, p.n_manning, H, z, z.copy(), p.sources, p.solid).to_f32_values())
    return out, gates


def run_ensemble(args, torch, swe, stream, rank, world, emit=True):
    """Batched ensemble: all of this rank's scenarios advance in one
    persistent launch per step (CUDA graph of K steps); ranks run disjoint
    scenarios (n each), value counts every rank's cells over the slowest
    rank's time."""
    n = int(args.workload.split("-")[1])
    probs, gates = flooded_ensemble(n, rank, world)
    cells = sum(p.params.nx * p.params.ny for p in probs)
    sols = [swe.Solver.from_problem(p, args.precision, stream=stream.cuda_stream) for p in probs]
    batch = swe.Batch(sols)
    seg = batch.autotune(2)
    # gate toggles inside the timed steps: each gate flips at its seeded step
    # of the run (steps are counted from the batch's creation; the timed
    # region starts after the untimed pass and the warm-up steps below)
    base = args.steps + args.warmup
    ev = [(k, int(i), int(j), base + int(st), 1 - int(c0)) for k, g in enumerate(gates)
          for i, j, c0, st in zip(g.ix, g.iy, g.closed0, g.toggle_step) if st < args.steps]
    if ev:
        batch.set_gate_events(*map(np.array, zip(*ev)))
    batch.step(args.steps, report=False)
    for _ in range(args.warmup):
        batch.step(1, report=False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        rank_barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        batch.step(args.steps, report=False)
        e1.record(stream)
        torch.cuda.synchronize()
        rank_barrier()
    ms = over_ranks(e0.elapsed_time(e1))
    infos = batch.step(0)
    batch.close()
    for x in sols:
        x.close()
    job_cells = over_ranks(cells, "sum")
    value = job_rate(job_cells * args.steps, ms)
    achieved = BYTES_PER_CELL[args.precision] * cells / (ms / args.steps * 1e-3) / 1e9
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = json.load(open(peaks_path))["hbm_gbs"] if os.path.exists(peaks_path) else 6800.0
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": args.workload, "scenarios": n * world, "scenarios_per_gpu": n,
                           "cells": int(job_cells),
                           "sizes": [min(p.params.nx for p in probs), max(p.params.nx for p in probs)],
                           "seg_h_autotuned": seg, "gates": int(sum(len(g.ix) for g in gates)),
                           "gate_toggles_in_timed_steps": len(ev),
                           "wet_cells_end": int(sum(i["wet_cells"] for i in infos)),
                           "l2": "inputs larger than L2",
                           "parallelism": f"scenarios sharded over {world} ranks" if world > 1 else "single GPU"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None, "kernel": "k_fused_batch<float>",
                             "algorithmic_bytes_per_cell": BYTES_PER_CELL[args.precision]},
                "cpu_baseline": None, "e2e": None, "gpu_launches": args.steps, "clocks": clk.summary()}
        if emit:
            print(json.dumps(line), flush=True)
        return line
    return None


# algorithmic FLOPs per pixel of the closure network (3x3 convolutions
# 5 -> 32 -> 32 -> 32 -> 3): forward, weight gradients, and data gradients
# of layers 1-3 (the input's gradient is not needed)
_CNN_CH = (5, 32, 32, 32, 3)
CNN_FWD_FLOP = sum(2 * 9 * a * b for a, b in zip(_CNN_CH[:-1], _CNN_CH[1:]))
CNN_TRAIN_FLOP = 3 * CNN_FWD_FLOP - 2 * 9 * _CNN_CH[0] * _CNN_CH[1]
# algorithmic HBM bytes per pixel of the forward pass: read the 16-channel
# BF16 input (32 B) and each hidden layer's 32 BF16 channels once (3 x 64 B),
# write the hidden layers (3 x 64 B) and the 3 FP32 outputs (12 B).  With 32
# channels a 3x3 layer does 144 FLOP per byte moved, below GB300's ridge
# point (~280), so the forward is bound by HBM, not the tensor cores.
CNN_FWD_BYTES = 32 + 3 * 64 + 3 * 64 + 12


def run_cnn(args, torch, swe, stream, rank, world, emit=True):
    """Closure network on one coarse grid (cnn-<n>sq: n x n pixels): K
    training steps (forward, backward, Adam) timed with CUDA events."""
    from paper_1705_00614_gb300 import closure
    n = int(args.workload.split("-")[1].replace("sq", ""))
    g = torch.Generator(device="cuda").manual_seed(1234)
    x = torch.zeros((1, n, n, 16), dtype=torch.bfloat16, device="cuda")
    x[..., :5] = torch.randn((1, n, n, 5), generator=g, device="cuda").to(torch.bfloat16)
    t = torch.randn((1, n, n, 3), generator=g, device="cuda")
    net = swe.CNN(1, n, n, stream=stream.cuda_stream)
    net.set_params(swe.flatten_cnn_params(closure.he_init(7)))
    for _ in range(args.warmup):
        net.train_step(x.data_ptr(), t.data_ptr(), 1e-4, report=False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        rank_barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            net.train_step(x.data_ptr(), t.data_ptr(), 1e-4, report=False)
        e1.record(stream)
        for _ in range(args.steps):
            net.forward(x.data_ptr())
        e2.record(stream)
        torch.cuda.synchronize()
        rank_barrier()
    ms_train = over_ranks(e0.elapsed_time(e1)) / args.steps
    ms_fwd = over_ranks(e1.elapsed_time(e2)) / args.steps
    net.close()
    px = n * n
    tflops = CNN_TRAIN_FLOP * px / (ms_train * 1e-3) / 1e12
    fwd_tflops = CNN_FWD_FLOP * px / (ms_fwd * 1e-3) / 1e12
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, src = (json.load(open(peaks_path))["bf16_tflops"], "measured") if os.path.exists(peaks_path) \
        else (1900.0, "fallback")
    hbm_peak = json.load(open(peaks_path))["hbm_gbs"] if os.path.exists(peaks_path) else 6800.0
    fwd_gbs = CNN_FWD_BYTES * px / (ms_fwd * 1e-3) / 1e9
    if rank == 0:
        line = {"metric": "closure CNN training throughput", "value": job_rate(world * px, ms_train),
                "unit": "Gpixel-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_train, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16", "data": "synthetic",
                "config": {"workload": args.workload, "pixels": px, "channels": list(_CNN_CH),
                           "train_flop_per_pixel": CNN_TRAIN_FLOP, "fwd_flop_per_pixel": CNN_FWD_FLOP,
                           "forward_ms": ms_fwd, "forward_tflops": fwd_tflops,
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                             "frac": tflops / peak, "peak_source": src, "traffic": None,
                             "kernel": "k_conv + k_wgrad_tc (tcgen05), BF16"},
                "forward_roofline": {"bound": "hbm", "achieved": fwd_gbs, "peak": hbm_peak, "unit": "GB/s",
                                     "frac": fwd_gbs / hbm_peak, "bytes_per_pixel": CNN_FWD_BYTES,
                                     "kernel": "k_conv x 4 (forward)"},
                "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk.summary()}
        if emit:
            print(json.dumps(line), flush=True)
        return line
    return None


# Short runs of the other measured paths that the default (one-GPU) run
# adds to its line: (workload, timed steps, warm-up steps, runner name)
SECONDARY = (("ensemble-64", 500, 3, "run_ensemble"), ("cnn-2048sq", 20, 5, "run_cnn"))
_SECONDARY_CONFIG = ("scenarios", "cells", "sizes", "gates", "gate_toggles_in_timed_steps", "pixels",
                     "forward_ms", "forward_tflops")


def secondary_entry(line):
    """The part of a secondary workload's line that the default line keeps."""
    out = {k: line[k] for k in ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "dtype",
                                "roofline", "forward_roofline", "gpu_launches", "clocks") if k in line}
    out["workload"] = line["config"]["workload"]
    out["config"] = {k: line["config"][k] for k in _SECONDARY_CONFIG if k in line["config"]}
    return out


def wants_secondary(args, world, default_workload):
    """The secondary runs belong to the default line only: one GPU, the
    default workload in FP32, the fused step without skipping, and not
    turned off with --no-secondary."""
    return (world == 1 and not args.no_secondary and args.workload == default_workload and args.precision == "f32"
            and args.mode == "fused" and not args.skip_dry)


def run_secondary(args, torch, swe):
    """Each secondary workload on a stream of its own; an exception becomes
    an entry with the error instead of a value."""
    out = []
    for wl, steps, warmup, fn in SECONDARY:
        a2 = argparse.Namespace(**vars(args))
        a2.workload, a2.steps, a2.warmup = wl, steps, warmup
        try:
            stream = torch.cuda.Stream()
            torch.cuda.set_stream(stream)
            line = globals()[fn](a2, torch, swe, stream, 0, 1, emit=False)
            torch.cuda.synchronize()
            out.append(secondary_entry(line))
        except Exception as e:  # report, do not lose the headline line
            out.append({"workload": wl, "error": f"{type(e).__name__}: {e}"[:300]})
    return out


def choose_on_validation(names, alphas, err_last, bar=0.01):
    """The closed variant the validation seeds pick: the largest correction
    scale whose mean relative error at the longest horizon stays within the
    bar (the most the network may act while meeting it); if none does, the
    one with the smallest error.  A diverged run (NaN) never passes; among
    equal scales the first listed wins."""
    err = {k: float(np.nan_to_num(err_last[k], nan=np.inf)) for k in names}
    ok = [(a, -i, k) for i, (k, a) in enumerate(zip(names, alphas)) if err[k] <= bar]
    if ok:
        return max(ok)[2]
    return min(names, key=lambda k: err[k])


def run_closure(args, torch, swe, stream, rank, world):
    """Learned closure of the 4x coarser grid (closure-<n>sq: fine n^2 at
    dx = 5 m, coarse (n/4)^2 at 20 m).  Trains the network on fine runs of
    the training seeds; runs the validation seeds fine, coarse plain and
    coarse closed with every candidate correction scale alpha side by side
    and keeps the alpha with the smallest mean error at the longest horizon;
    then runs the held-out test seeds the same way and reports the relative
    L2 error in H of the plain and the closed coarse runs against the
    restricted fine solution at several horizons (the chosen alpha's test
    errors are the line's value), and the wall-clock speed-up of the closed
    coarse solve over the fine solve (same simulated time).  The three seed
    sets are disjoint; nothing is chosen on the test seeds."""
    from paper_1705_00614_gb300 import closure as CL
    n = int(args.workload.split("-")[1].replace("sq", ""))
    tau_c = 0.2
    train_seeds = list(range(20000, 20000 + args.closure_train))
    test_seeds = list(range(20064, 20064 + args.closure_test))
    val_seeds = list(range(20100, 20100 + args.closure_val))
    assert not (set(train_seeds) & set(test_seeds)) and not (set(val_seeds) & (set(train_seeds) | set(test_seeds)))
    horizons = [h for h in (10, 100, 1000, 5000) if h <= args.closure_steps]

    def scenario(seed):
        return CL.dam_release(I.floodplain(n, 5.0, seed, seed + 1, nsrc=20,
                                           hydro=I.Hydrograph(0, 2.0, 40.0, 20.0)))

    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    win = args.closure_window
    # input and target statistics from the first training seeds' runs
    norm = CL.estimate_norm(torch, [scenario(sd) for sd in train_seeds[:4]], 40 * win, tau_c, rng, 128,
                            bed=args.closure_bed, horizon=win, stride=args.closure_stride)
    X, T = [], []
    for sd in train_seeds:
        x, t = CL.collect(torch, scenario(sd), args.closure_collect, tau_c, norm.inp(), norm.out(),
                          args.closure_crops, 128, rng, stream=stream.cuda_stream, noise=args.closure_noise,
                          bed=args.closure_bed, horizon=win, stride=args.closure_stride)
        X.append(x)
        T.append(t)
    X = torch.cat(X)
    T = torch.cat(T)
    params, hist = CL.train(torch, X, T, args.closure_iters, 16, 1e-3, 1, stream=stream.cuda_stream, log_every=500)
    # optional rounds of pairs from the closed model's own trajectory
    for r in range(args.closure_dagger):
        for sd in train_seeds:
            x, t = CL.collect_closed(torch, scenario(sd), args.closure_collect, tau_c, params, norm,
                                     args.closure_crops, 128, rng, stream=stream.cuda_stream, bed=args.closure_bed,
                                     stride=args.closure_stride, bound=args.closure_bound)
            if x is not None:
                X = torch.cat([X, x])
                T = torch.cat([T, t])
        params, h2 = CL.train(torch, X, T, args.closure_iters // 2, 16, 5e-4, 2 + r, stream=stream.cuda_stream,
                              log_every=500, init=params)
        hist += h2
    del X, T
    t_train = time.perf_counter() - t0

    # candidate scales: "a" scales every correction by a; "a/m" keeps only
    # the momentum corrections (scaled by a), the depth correction off
    specs = [(float(x.split("/")[0]), 0.0 if x.endswith("/m") else None) for x in args.closure_alpha.split(",")]
    alphas = [a for a, _ in specs]
    names = ["plain"] + [f"closed_a{a:g}" + ("_momentum_only" if ah == 0.0 else "") for a, ah in specs]
    ms_fine, ms_closed = [], []

    def run_seeds(seeds):
        errs = {k: {h: [] for h in horizons} for k in names}
        for sd in seeds:
            fp = scenario(sd)
            cp = CL.coarse_problem(fp, args.closure_bed)
            fine = swe.Solver.from_problem(CL.with_dt(fp, tau_c / 4.0), "f32", stream=stream.cuda_stream)
            plain = swe.Solver.from_problem(CL.with_dt(cp, tau_c), "f32", stream=stream.cuda_stream)
            closed = [swe.Solver.from_problem(CL.with_dt(cp, tau_c), "f32", stream=stream.cuda_stream)
                      for _ in alphas]
            ref = swe.Solver.from_problem(CL.with_dt(cp, tau_c), "f32", stream=stream.cuda_stream)
            nets = [swe.CNN(1, cp.params.ny, cp.params.nx, stream.cuda_stream) for _ in alphas]
            alive = [True] * len(alphas)
            try:
                plain.restrict_from(fine)
                for c, net, (a, ah) in zip(closed, nets, specs):
                    net.set_params(params)
                    c.restrict_from(fine)
                    c.attach_closure(net, CL.shrink(norm, a, ah).all())
                    c.closure_bound(args.closure_bound)
                done = 0
                for h in horizons:
                    k = h - done
                    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                    e[0].record(stream)
                    fine.step(4 * k, report=False)
                    e[1].record(stream)
                    if alive[0]:
                        closed[0].step_closed(k, report=False)
                    e[2].record(stream)
                    for q in range(1, len(alphas)):
                        if alive[q]:
                            closed[q].step_closed(k, report=False)
                    plain.step(k, report=False)
                    torch.cuda.synchronize()
                    ms_fine.append(e[0].elapsed_time(e[1]) / k)
                    if alive[0]:
                        ms_closed.append(e[1].elapsed_time(e[2]) / k)
                    done = h
                    ref.restrict_from(fine)
                    Hr = ref.get_state()[0]
                    den = max(np.linalg.norm(Hr), 1e-30)
                    errs["plain"][h].append(float(np.linalg.norm(plain.get_state()[0] - Hr) / den))
                    for q, (c, a) in enumerate(zip(closed, alphas)):
                        Hc = c.get_state()[0] if alive[q] else None
                        if Hc is None or not np.isfinite(Hc).all():
                            alive[q] = False  # diverged: reported as NaN from here on
                            errs[names[1 + q]][h].append(float("nan"))
                        else:
                            errs[names[1 + q]][h].append(float(np.linalg.norm(Hc - Hr) / den))
            finally:
                for c in closed:
                    c.attach_closure(None, norm.all())
                for x in [fine, plain, ref] + closed + nets:
                    x.close()
        return {k: {h: float(np.mean(v)) for h, v in d.items()} for k, d in errs.items()}

    last = horizons[-1]
    val = run_seeds(val_seeds)
    chosen = choose_on_validation(names[1:], alphas, {k: val[k][last] for k in names[1:]})
    test = run_seeds(test_seeds)
    gain = [h for h in horizons if test[chosen][h] < test["plain"][h]]
    speedup = float(np.median(ms_fine)) / float(np.median(ms_closed))
    if rank == 0:
        line = {"metric": "CNN-closure vs fine solve: relative L2 error in H", "value": test[chosen][last],
                "unit": "fraction", "n_gpus": world, "steps": last, "warmup": 0,
                "ms_per_step": float(np.median(ms_closed)), "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
                "config": {"workload": args.workload, "fine": f"{n}^2 dx 5 m", "coarse": f"{n // 4}^2 dx 20 m",
                           "scenario": "fractal floodplain, flood release (+2 m over the first quarter) and inflow",
                           "tau_coarse_s": tau_c, "train_seeds": len(train_seeds), "val_seeds": len(val_seeds),
                           "test_seeds": len(test_seeds), "collect_steps_per_seed": args.closure_collect,
                           "target_window_steps": win, "window_stride_steps": args.closure_stride,
                           "crops_per_window": args.closure_crops,
                           "train_iters": args.closure_iters,
                           "dagger_rounds": args.closure_dagger, "input_noise": args.closure_noise,
                           "coarse_bed": args.closure_bed, "correction_bound": args.closure_bound,
                           "final_train_loss": hist[-1][1], "train_wall_s": t_train,
                           "rel_l2_test": test, "rel_l2_val": val, "chosen_on_val": chosen,
                           "closed_below_plain_at": gain,
                           "target": 0.01, "speedup_closed_coarse_vs_fine": speedup,
                           "ms_per_fine_step": float(np.median(ms_fine)),
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None}
        print(json.dumps(line), flush=True)


def run_nest(args, torch, swe, stream, rank, world):
    """Two-level nesting (nest-<n>sq): a flooded n^2 floodplain at dx = 20 m
    with an n^2 patch at 5 m over its central (n/4)^2 coarse cells; K nested
    coarse steps (each: one coarse step, four fine sub-steps with ghost
    fills, feedback) timed with CUDA events.  value counts every cell update
    of both levels."""
    from paper_1705_00614_gb300 import closure as CL
    n = int(args.workload.split("-")[1].replace("sq", ""))
    # one fine terrain under both levels: the coarse bed is its 4 x 4 means
    # over the patch and the coarse generator's elsewhere
    base = I.floodplain(n, 20.0, 2031, 2032, nsrc=1)
    eta0 = float(np.median(base.b))
    ix0 = iy0 = 3 * n // 8
    fine_full = I.floodplain(n + 2 * 10, 5.0, 2033, 2034, nsrc=1)
    bf_ext = fine_full.b - np.median(fine_full.b) + eta0  # fine relief around the same water level
    nf_ext = fine_full.n_manning
    bf = bf_ext[10:10 + n, 10:10 + n]
    bc = base.b.copy()
    bc[iy0:iy0 + n // 4, ix0:ix0 + n // 4] = bf.reshape(n // 4, 4, n // 4, 4).mean(axis=(1, 3))
    Hc = np.maximum(0.0, eta0 - bc)
    z = np.zeros_like(Hc)
    pc = I.Params(**{**base.params.__dict__, "dt_fixed": 0.2})
    coarse = I.Problem("nest-coarse", pc, bc, base.n_manning, Hc, z, z.copy(), I.Sources.empty()).to_f32_values()
    Hf = np.maximum(0.0, eta0 - bf)
    zf = np.zeros_like(Hf)
    pf = I.Params(**{**fine_full.params.__dict__, "nx": n, "ny": n, "dt_fixed": 0.05})
    fine = I.Problem("nest-fine", pf, bf, nf_ext[10:10 + n, 10:10 + n], Hf, zf, zf.copy(),
                     I.Sources.empty()).to_f32_values()
    c = swe.Solver.from_problem(coarse, args.precision, stream=stream.cuda_stream)
    f = swe.Solver.from_problem(fine, args.precision, stream=stream.cuda_stream, ghost_ring=True)
    f.set_terrain_ext(np.asarray(bf_ext, np.float32).astype(np.float64),
                      np.asarray(nf_ext, np.float32).astype(np.float64))
    f.set_state(fine.H, fine.Qx, fine.Qy, 0.0)
    nest = swe.Nest(c, f, ix0, iy0)
    for _ in range(args.warmup):
        nest.step(1, report=False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        rank_barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        nest.step(args.steps, report=False)
        e1.record(stream)
        torch.cuda.synchronize()
        rank_barrier()
    ms = over_ranks(e0.elapsed_time(e1)) / args.steps
    ic, jf = nest.step(0)
    nest.close()
    c.close()
    f.close()
    updates = n * n + 4 * n * n
    if rank == 0:
        line = {"metric": "nested Gcell-updates/s (coarse + 4 fine sub-steps)",
                "value": job_rate(world * updates, ms), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": args.workload, "coarse": f"{n}^2 dx 20 m", "patch": f"{n}^2 dx 5 m",
                           "patch_origin_coarse": [ix0, iy0], "cell_updates_per_step": updates,
                           "coarse_wet_end": ic["wet_cells"], "fine_wet_end": jf["wet_cells"],
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def crop(prob, y0, x0, n):
    s = prob.sources
    keep = (s.ix >= x0) & (s.ix < x0 + n) & (s.iy >= y0) & (s.iy < y0 + n)
    src = I.Sources(s.ix[keep] - x0, s.iy[keep] - y0, s.weight[keep], s.vx[keep], s.vy[keep], s.hydro[keep],
                    s.hydrographs)
    par = I.Params(**{**prob.params.__dict__, "nx": n, "ny": n})
    sl = (slice(y0, y0 + n), slice(x0, x0 + n))
    return I.Problem("crop", par, prob.b[sl].copy(), prob.n_manning[sl].copy(), prob.H[sl].copy(),
                     prob.Qx[sl].copy(), prob.Qy[sl].copy(), src)


class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def alu_roofline(prof, cells, ms_per_step, nsm, clocks):
    """Instruction-issue roofline: one warp instruction per scheduler per
    cycle, four schedulers per SM."""
    mhz = clocks.get("sm_mhz")
    if prof is None or not mhz:
        return None
    achieved = prof["inst"] * cells / (ms_per_step * 1e-3) / 1e9
    peak = nsm * 4 * mhz * 1e6 / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G warp-instructions/s",
            "frac": achieved / peak, "inst_per_cell": prof["inst"],
            "peak_basis": f"{nsm} SMs x 4 schedulers x {mhz:.0f} MHz (median sampled SM clock)"}


def profile_per_cell(workload):
    """DRAM bytes and warp instructions per cell of the fused kernel from
    the committed ncu summary, if it was taken on the current kernel
    sources (else None)."""
    path = os.path.join(ROOT, "profiles", "k_fused_f32_dram.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_sources_sha256_16") != kernel_hash():
        return None
    try:
        return {"dram": float(kv["dram_bytes_per_cell"]), "inst": float(kv["warp_inst_per_cell"])}
    except (KeyError, ValueError):
        return None


def oracle_rate(prob, steps, cells_hint=None):
    import oracle
    oracle.build()
    bd = oracle._Bound(prob)
    H, Qx, Qy, t = prob.H, prob.Qx, prob.Qy, 0.0
    t0 = time.perf_counter()
    for _ in range(steps):
        H, Qx, Qy, info, _ = oracle.step(prob, H, Qx, Qy, t, bound=bd)
        t = info["t_new"]
    dt = time.perf_counter() - t0
    cells = prob.params.nx * prob.params.ny * steps
    return cells / dt / 1e9, dt


_BARRIER = None


def _oracle_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(job):
    prob, steps = job
    import oracle
    bd = oracle._Bound(prob)
    H, Qx, Qy, t = prob.H, prob.Qx, prob.Qy, 0.0
    _BARRIER.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        H, Qx, Qy, info, _ = oracle.step(prob, H, Qx, Qy, t, bound=bd)
        t = info["t_new"]
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate_procs(prob, steps, procs):
    """The oracle as it stands on `procs` host cores at once: one spawned
    process per core, all on the same crop, started together by a barrier.
    Returns (all processes' cell-updates / the slowest one's time, in G/s;
    that time in s)."""
    import oracle
    oracle.build()
    if procs <= 1:
        return oracle_rate(prob, steps)
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    with ctx.Pool(procs, initializer=_oracle_init, initargs=(barrier,)) as pool:
        dts = pool.map(_oracle_worker, [(prob, steps)] * procs)
    dt = max(dts)
    return prob.params.nx * prob.params.ny * steps * procs / dt / 1e9, dt


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, on crops of the workload."""
    if rank != 0:
        return
    prob, eta0 = flooded_workload(args.workload)
    n = args.ref_crop
    y0 = int(prob.sources.iy.min()) - n // 2
    c = crop(prob, max(0, y0), 0, n)
    procs = args.cpu_procs or host_cores()
    oracle_rate(c, args.warmup)
    val, dt = oracle_rate_procs(c, args.steps, procs)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "sample": f"{n}x{n} crop at the inflow strip",
                       "parallelism": f"{procs} host cores, one oracle process each"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": f"{args.steps} oracle steps of a {n}x{n} crop of {args.workload} "
                                       f"in each of {procs} processes"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="floodplain-16384sq-dx2m-flooded")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-crop", type=int, default=1024)
    ap.add_argument("--cpu-steps", type=int, default=20)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="oracle processes for the CPU baseline and the reference arm (0 = one per host core)")
    ap.add_argument("--skip-dry", action="store_true",
                    help="skip dry work items (the paper's K1 wet-block test); off for the headline")
    ap.add_argument("--seg-h", type=int, default=0, help="output rows per work item (0 = automatic)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="default workload: leave out the short ensemble and closure-network runs")
    ap.add_argument("--mode", default="fused", choices=["fused", "staged"],
                    help="staged: one kernel per stage (the paper's K2-K8 split), for per-stage time shares")
    ap.add_argument("--closure-train", type=int, default=64, help="closure workload: training seeds")
    ap.add_argument("--closure-val", type=int, default=8,
                    help="closure workload: validation seeds (choose the correction scale)")
    ap.add_argument("--closure-test", type=int, default=16, help="closure workload: held-out test seeds")
    ap.add_argument("--closure-collect", type=int, default=100, help="closure workload: coarse steps per seed")
    ap.add_argument("--closure-crops", type=int, default=4,
                    help="closure workload: 128^2 training crops per target window")
    ap.add_argument("--closure-stride", type=int, default=50,
                    help="closure workload: coarse steps between training windows (spreads the pairs over the run)")
    ap.add_argument("--closure-window", type=int, default=1,
                    help="closure workload: coarse steps per training target (average correction over the window)")
    ap.add_argument("--closure-iters", type=int, default=6000, help="closure workload: Adam steps")
    ap.add_argument("--closure-bound", type=float, default=0.5,
                    help="closure workload: corrections bounded by this fraction of the plain flux sums (0: unbounded)")
    ap.add_argument("--closure-steps", type=int, default=5000, help="closure workload: longest horizon")
    ap.add_argument("--closure-alpha", default="1,0.5,0.25,0.1,0.05",
                    help="closure workload: comma-separated correction scales (a suffix /m keeps the momentum "
                         "corrections only); the validation seeds pick one")
    ap.add_argument("--closure-bed", default="volume", choices=["mean", "volume"],
                    help="closure workload: coarse bed from 4x4 means, or volume-matched in partly wet cells")
    ap.add_argument("--closure-noise", type=float, default=0.0,
                    help="closure workload: relative input noise on the coarse states the training pairs start from")
    ap.add_argument("--closure-dagger", type=int, default=0,
                    help="closure workload: rounds of training pairs from the closed model's own trajectory")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    barrier = rank_barrier

    from paper_1705_00614_gb300 import build as B
    from paper_1705_00614_gb300 import swe
    B.build()

    if args.workload.startswith("nest-"):
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        run_nest(args, torch, swe, stream, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return

    if args.workload.startswith("closure-"):
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        run_closure(args, torch, swe, stream, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return

    if args.workload.startswith("cnn-"):
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        run_cnn(args, torch, swe, stream, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return

    if args.workload.startswith("ensemble-"):
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        run_ensemble(args, torch, swe, stream, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return

    prob, eta0 = flooded_workload(args.workload)
    cells = prob.params.nx * prob.params.ny
    # a dedicated (non-default) stream: the library launches on it and the
    # CUDA events below are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    solver = swe.Solver.from_problem(prob, args.precision, mode=args.mode, stream=stream.cuda_stream,
                                     seg_h=args.seg_h, skip_dry=args.skip_dry)

    # instantiate the CUDA graph of K steps once, restart, then W untimed
    # single-launch warm-up steps (they leave the cached K-step graph alone)
    solver.step(args.steps, report=False)
    solver.set_state(prob.H, prob.Qx, prob.Qy, 0.0)
    for _ in range(args.warmup):
        solver.step(1, report=False)
    torch.cuda.synchronize()

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        solver.step(args.steps, report=False)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = over_ranks(e0.elapsed_time(e1))
    info = solver.step(0)
    ms_per_step = ms / args.steps
    value = job_rate(world * cells * args.steps, ms)

    # end to end through the C ABI with pinned host buffers: the state in its
    # own precision (swe_set_state_native / swe_get_state_native), and for
    # comparison the FP64 host arrays of swe_set_state / swe_get_state
    shape = (prob.params.ny, prob.params.nx)

    def e2e_leg(tdt, native):
        hb = [torch.empty(shape, dtype=tdt, pin_memory=True).numpy() for _ in range(6)]
        hb[0][...] = prob.H
        hb[1][...] = prob.Qx
        hb[2][...] = prob.Qy
        up = solver.set_state_native if native else solver.set_state
        down = solver.get_state_native_into if native else solver.get_state_into
        up(hb[0], hb[1], hb[2], 0.0)
        solver.step(1)
        down(hb[3], hb[4], hb[5])
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            up(hb[0], hb[1], hb[2], 0.0)
            solver.step(1, report=False)
            down(hb[3], hb[4], hb[5])
        torch.cuda.synchronize()
        e2e_s = over_ranks(time.perf_counter() - t0)
        del hb
        return job_rate(world * cells * args.e2e_steps, e2e_s * 1e3), 3 * cells * (4 if tdt == torch.float32 else 8)

    state_dt = torch.float32 if args.precision == "f32" else torch.float64
    e2e_val, io_bytes = e2e_leg(state_dt, True)
    # the FP64-host comparison pins another 12.9 GB per process: one GPU only
    if args.precision == "f32" and world == 1:
        e2e64_val, io64_bytes = e2e_leg(torch.float64, False)
    elif args.precision == "f32":
        e2e64_val, io64_bytes = None, 3 * cells * 8
    else:
        e2e64_val, io64_bytes = e2e_val, io_bytes

    bpc = BYTES_PER_CELL[args.precision]
    achieved = bpc * cells / (ms_per_step * 1e-3) / 1e9
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak = json.load(open(peaks_path))["hbm_gbs"]
        peak_src = "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    prof = profile_per_cell(args.workload) if args.precision == "f32" else None
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    solver.close()

    no_roof = args.skip_dry or args.mode == "staged"
    if rank == 0:
        cpu = None
        if not args.no_cpu:
            n = args.ref_crop
            y0 = int(prob.sources.iy.min()) - n // 2
            c = crop(prob, max(0, y0), 0, n)
            procs = args.cpu_procs or host_cores()
            val, dt = oracle_rate_procs(c, args.cpu_steps, procs)
            cpu = {"value": val, "unit": UNIT, "cores": procs, "kind": "oracle",
                   "sample": f"{args.cpu_steps} FP64 oracle steps of a {n}x{n} crop at the inflow strip in each "
                             f"of {procs} processes, one per host core ({dt:.1f} s)"}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": args.workload, "cells": cells, "dx_m": prob.params.dx,
                           "initial_eta_m": None if eta0 is None else round(eta0, 4),
                           "wet_fraction": float((prob.H > prob.params.eps).mean()),
                           "skip_dry": args.skip_dry, "seg_h": args.seg_h or "auto",
                           "skipped_items_last_step": info["skipped"],
                           # H, Qx, Qy, b, n and the two stored accelerations
                           "l2": f"inputs larger than L2 ({7 * cells * (4 if args.precision == 'f32' else 8) / 1e9:.1f} GB read per step)",
                           "parallelism": "replicas" if world > 1 else "single GPU", "mode": args.mode,
                           "final_t_s": info["t"], "wet_cells_end": info["wet_cells"]},
                "roofline": {"bound": "hbm", "achieved": None if no_roof else achieved, "peak": peak,
                             "unit": "GB/s", "frac": None if no_roof else achieved / peak,
                             "peak_source": peak_src, "nominal_peak": NOMINAL_HBM_GBS,
                             "frac_nominal": None if no_roof else achieved / NOMINAL_HBM_GBS,
                             "note": ("skip_dry: skipped items move (almost) no state, so the method's 32 B per "
                                      "counted cell-update does not apply") if args.skip_dry else
                                     ("staged: one kernel per stage, every intermediate in HBM; see the launch "
                                      "list for per-stage times") if args.mode == "staged" else None,
                             "traffic": None if prof is None else prof["dram"] * cells,
                             "kernel": f"k_fused<{'float' if args.precision == 'f32' else 'double'}>",
                             "algorithmic_bytes_per_cell": bpc},
                "alu_roofline": None if no_roof else alu_roofline(prof, cells, ms_per_step, nsm, clk.summary()),
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
                        "host_dtype": args.precision, "fp64_host": {"value": e2e64_val, "unit": UNIT,
                                                                   "h2d_bytes_per_step": io64_bytes,
                                                                   "d2h_bytes_per_step": io64_bytes}},
                "gpu_launches": args.steps * (1 if args.mode == "fused" else 12 + (1 if len(prob.sources) else 0)),
                "clocks": clk.summary()}
        if wants_secondary(args, world, ap.get_default("workload")):
            line["secondary"] = run_secondary(args, torch, swe)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
