"""Benchmark: proton-iterations/s of the fused MLP + DROP projection on GB300.

Default workload: 1e9 synthetic histories on a 200x200x48 grid of
1 x 1 x 2 mm voxels (1.92M voxels), a seeded random head phantom, 90
projection angles, 50 DROP blocks (``--workload head200``). ``--workload
head`` is the 50M-history head on a 160x160x64 grid of 1.25 mm voxels (1.64M
voxels), 10 blocks. One step = one DROP sweep over all histories (every
block's fused MLP + projection kernel and its apply); value = histories x
sweeps / time with the records resident in HBM.
e2e = the same metric for a full 10-sweep reconstruction through the public
API from pinned host buffers (load + validation + block counts + 10 sweeps +
copy of x back to the host). time_to_image = the metric's second half: the
seconds to <= 1 % (and 0.6 %) mean RSP error of the plain and of the
warm-started solver on held-out 1e9-history heads, the network trained in
the same run (time_to_image(); --no-time-to-image skips it). ``--workload
tiny`` is the 100k-history 32^3 water cylinder.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the reference arm: there is
no reference code to run, only the paper) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "proton-iterations/s (fused MLP+projection)"
UNIT = "proton-iterations/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.rows = []
        self._p = None
        self._t = None

    def start(self):
        try:
            self._p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                        "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                       stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self._p = None
            return

        def rd():
            for line in self._p.stdout:
                self.rows.append([x.strip() for x in line.split(",")])

        self._t = threading.Thread(target=rd, daemon=True)
        self._t.start()

    def stop(self):
        if self._p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self._p.terminate()
        try:
            self._p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self._p.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ALU roof: FP32/INT32 lanes per SM x SMs x maximum SM clock (recipe unit counts)
ALU_LANES_PER_SM = 128
N_SMS = 152
OPS_PER_MLP_NODE = 27  # t/v 8, rotation 4, grid 3, scale 3, rounding 3, floor 3, crossing test 3
OPS_PER_RUN = 11  # crossing fraction 3, accumulation 2, index 3, load/atomic 3


# the sources the fused kernel is compiled from
FUSED_SOURCES = ("pct_internal.h", "pct_walk.cuh", "pct_drop.cuh", "pct_kernels.cu")


def strip_c_comments(text: str) -> str:
    """C/C++/CUDA source without its comments and with runs of white space
    collapsed to one blank (string and character literals kept as written)."""
    out, i, n = [], 0, len(text)
    while i < n:
        ch = text[i]
        if ch in "\"'":
            j = i + 1
            while j < n and text[j] != ch:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(ch)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash(read=None) -> str:
    """Hash of the fused kernel's CUDA sources, comments and layout aside:
    counters taken on other code are stale. read(name) returns a file's text
    (default: the working tree)."""
    import hashlib

    d = os.path.join(ROOT, "paper_1707_05014_gb300", "csrc")
    if read is None:
        def read(name):
            with open(os.path.join(d, name), encoding="utf-8") as fh:
                return fh.read()
    h = hashlib.sha256()
    for f in FUSED_SOURCES:
        h.update(f.encode())
        h.update(strip_c_comments(read(f)).encode())
    return h.hexdigest()[:16]


def traffic_per_launch(cnt, args, per_block):
    """DRAM bytes of one fused launch from the committed counters, or None
    unless they were taken on this configuration: the one-lane kernel without
    a hull, the same workload and the same histories per launch."""
    same = (cnt is not None and args.lanes <= 1 and not args.hull and args.workload == cnt.get("workload")
            and per_block == cnt.get("histories"))
    return cnt["dram_bytes_per_history"] * per_block if same else None


def ncu_counters():
    """DRAM bytes per history of the fused kernel from the committed ncu summary,
    if it was taken on the current kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "drop_fused_head200_counters.json")) as f:
            c = json.load(f)
    except OSError:
        return None
    return c if c.get("source_hash") == kernel_source_hash() else None


def _cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_sample(wl, n_sample: int):
    """n_sample histories of the workload, generated on the host with the same
    recipe (a different seed stream from the GPU set)."""
    from paper_1707_05014_gb300 import synthetic as S

    return S.make_histories(wl, n=n_sample, seed_offset=777)


def oracle_rate(wl, rec, sweeps: int = 1, node_step: float = 0.0, threads: int = 1):
    """Time the FP64 CPU oracle's DROP on the host histories `rec`: single
    thread (threads = 1) or each block's histories split over `threads`
    OpenMP threads (0: all host cores). Returns (rate, seconds, threads)."""
    import oracle as O

    O.build()
    n = len(rec["t0"])
    t = time.perf_counter()
    if threads == 1:
        O.drop(wl.grid, rec, wl.n_blocks, sweeps, mode=O.MODE_FP32, node_step=node_step)
    else:
        O.drop_threads(wl.grid, rec, wl.n_blocks, sweeps, threads=threads, mode=O.MODE_FP32, node_step=node_step)
    dt = time.perf_counter() - t
    return n * sweeps / dt, dt, (1 if threads == 1 else (threads or O.max_threads()))


def run_reference(args):
    """Reference arm: the oracle as it stands, on the host cores, on bounded
    samples of the same workload (one sweep of ``--ref-sample`` histories per
    step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1707_05014_gb300 import synthetic as S

    wl = main_workload(args)
    rec = oracle_sample(wl, args.ref_sample)
    rates = []
    cores = 1
    for i in range(args.warmup + args.steps):
        r, dt, cores = oracle_rate(wl, rec, threads=0)
        if i >= args.warmup:
            rates.append((r, dt))
    total_units = args.ref_sample * len(rates)
    total_t = sum(dt for _, dt in rates)
    value = total_units / total_t
    sample = (f"{args.ref_sample} histories of the {wl.name} workload, 1 sweep, {wl.n_blocks} blocks, per step; "
              f"FP64 oracle, each block's histories split over {cores} OpenMP threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / len(rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "grid": grid_text(wl.grid), "histories": wl.n, "n_blocks": wl.n_blocks,
                   "sample_histories": args.ref_sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main_workload(args, rank: int = 0):
    """The throughput workload: head200 (1e9 histories, 200x200x48 @ 1x1x2 mm,
    50 blocks), head (50M histories, 160x160x64 @ 1.25 mm, 10 blocks) or tiny
    (100k histories, 32^3 @ 2 mm, water cylinder, 10 blocks); each rank draws
    its own reconstruction (weak scaling)."""
    from paper_1707_05014_gb300 import synthetic as S

    if args.workload == "head":
        wl = S.head_workload(args.n or 50_000_000, seed=2 + rank)
    elif args.workload == "tiny":
        wl = S.tiny_workload(args.n or 100_000, seed=1 + rank)
    else:
        wl = S.head200_workload(args.n or 1_000_000_000, seed=5 + rank)
    return dataclasses.replace(wl, n_blocks=args.blocks) if args.blocks else wl


def grid_text(g) -> str:
    return f"{g.nx}x{g.ny}x{g.nz} @ {g.hx:g}x{g.hy:g}x{g.hz:g} mm ({g.m / 1e6:.2f}M voxels)"


def max_over_ranks(ms: float, device=None) -> float:
    """The slowest rank's time (the job's time): all-reduce MAX when a process
    group is up, else the local value."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_batched(args):
    """Batched variant: 32 independent reconstructions of uneven size advanced
    together (pct_batch_*) in the mode the autotuner picks (graph branches of
    the per-block kernels, or one persistent launch per sweep); the same sweep
    done one context at a time (pct_iterate) is timed beside it."""
    import torch

    from paper_1707_05014_gb300 import build as B
    from paper_1707_05014_gb300 import pct as P
    from paper_1707_05014_gb300 import synthetic as S

    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    B.build()
    wls = S.batch_workloads(n_recon=args.n_recon, seed=4 + rank)
    ctxs, ops_per_sweep, total = [], 0.0, 0
    for w in wls:
        rec = S.make_histories_device(w, device=f"cuda:{local}")
        c = P.Context(w.grid, n_blocks=w.n_blocks, device=local)
        c.load(rec)
        k = min(w.n, 20_000)
        rs = P.Context(w.grid, n_blocks=1, device=local)
        rs.load({f: v[:k] for f, v in rec.items()})
        runs = float(rs.rows(0, k)[0][-1].item()) / k
        rs.close()
        del rec
        ops_per_sweep += w.n * (OPS_PER_MLP_NODE * (c.K + 1) + OPS_PER_RUN * runs)
        total += w.n
        ctxs.append(c)
    torch.cuda.empty_cache()

    def sweep_ms(**kw):
        """ms per batched sweep (after one warm-up sweep) of one batch mode."""
        with P.Batch(ctxs, **kw) as bb:
            bb.iterate(1)
            bb.sync()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(torch.cuda.current_stream())
            bb.iterate(2)
            a1.record(torch.cuda.current_stream())
            bb.sync()
            return a0.elapsed_time(a1) / 2

    # both modes at their defaults, measured side by side (the sweeps change x,
    # which does not change the work of a sweep)
    modes = {"persistent_ms": sweep_ms(mode=P.BATCH_PERSISTENT), "graph_branches_ms": sweep_ms(mode=P.BATCH_GRAPH_BRANCHES),
             "graph_branches_32_lanes_ms": sweep_ms(mode=P.BATCH_GRAPH_BRANCHES, lanes=32)}
    batch = P.Batch(ctxs)
    tune = batch.autotune()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.iterate(1)
    batch.sync()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = batch.launches
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        batch.iterate(1)
    e1.record(stream)
    batch.sync()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = batch.launches - l0
    # the same sweeps one reconstruction at a time (pct_iterate, one graph each)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for c in ctxs:
        c.iterate(1)
    s1.record(stream)
    torch.cuda.synchronize()
    seq_ms = s0.elapsed_time(s1)
    batch.close()
    value = total * args.steps * world / (ms / 1e3)
    alu_peak = ALU_LANES_PER_SM * N_SMS * _peaks()[0].get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = ops_per_sweep * args.steps / (ms / 1e3) / 1e12
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched{len(wls)}", "reconstructions": len(wls), "histories": total,
                       "grids": "64x64x32 .. 160x160x64 over 200 mm", "histories_each": "2M-40M log-uniform",
                       "n_blocks": 10,
                       "step": "one DROP sweep of every reconstruction (" + (
                           "one persistent launch" if tune.get("mode") == "persistent" else
                           f"graph of {tune.get('branches')} branches of per-block launches") + ")",
                       "parallelism": f"replicas{world}"},
            "roofline": {"kernel": "batch_kernel" if tune.get("mode") == "persistent" else (
                             "drop_group_kernel" if tune.get("lanes", 1) > 1 else "drop_fused_kernel"), "bound": "alu", "achieved": achieved, "peak": alu_peak,
                         "unit": "Tops/s", "frac": achieved / alu_peak, "traffic": None},
            "autotune": tune, "modes_ms_per_sweep": modes, "sequential_contexts_value": total / (seq_ms / 1e3),
            "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    return 0


def run_precision(args):
    """Precision variant: 250M histories on the head grid, 40 blocks, 8 sweeps
    (FP32 fused MLP + projection with Kahan a_i.x, FP64 MLP tables), timed.
    The error of every stage against the FP64 oracle on a 1M-history subset
    (nodes, index lists and chords, a_i.x with and without Kahan, the image
    after the 8 sweeps) is test infrastructure: tests/precision_report.py."""
    import torch

    from paper_1707_05014_gb300 import build as B
    from paper_1707_05014_gb300 import pct as P
    from paper_1707_05014_gb300 import synthetic as S

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    B.build()
    n_full = args.n or 250_000_000
    base = S.head_workload(n_full, seed=3)
    wl = S.Workload(f"head160_precision_{n_full}", base.grid, n_full, 3, 90, base.t_range, base.v_range, 40, 8,
                    "head")
    g = wl.grid
    rec = S.make_histories_device(wl, device=f"cuda:{local}")
    ctx = P.Context(g, n_blocks=40, flags=P.FLAG_PROFILE, device=local)
    ctx.load(rec, borrow=True)
    del rec
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    ctx.iterate(1)
    ctx.last_sweep_times()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        ctx.iterate(1)
        ctx.last_sweep_times()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ctx.close()
    value = wl.n * args.steps / (ms / 1e3)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "grid": "160x160x64 @ 1.25 mm", "histories": wl.n, "n_blocks": 40,
                   "step": "one DROP sweep", "kahan": True, "mlp_table": "fp64 on GPU"},
        "precision": "error budget against the FP64 oracle: python tests/precision_report.py", "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def time_to_image(args, local: int, log) -> dict:
    """Learned warm start against the plain solver: 200 plain-solver
    reconstructions of seeded random heads (200x200x48 grid, 1x1x2 mm) train
    the network; on held-out heads with 1e9 histories, the time to each target
    mean RSP error of the warm-started solve and of the plain solver (CUDA
    events on the GPU work; the error check against the known phantom is
    outside the timed region). Both solvers use the same block count (--ws-blocks,
    or tuned for the plain solver with --ws-tune-blocks); a study of the plain
    solver over several block counts is reported beside it. Each timed solve
    starts from a fresh load with the block weights formed beforehand
    (pct_block_weights, timed separately): the clock starts at the first
    sweep with the records resident. Every step runs in the library's
    kernels."""
    import numpy as np
    import torch

    from paper_1707_05014_gb300 import pct as P
    from paper_1707_05014_gb300 import synthetic as S
    from paper_1707_05014_gb300 import warmstart as W

    g = W.training_grid()
    targets = sorted({args.ws_target, *([args.ws_target2] if args.ws_target2 > 0 else [])}, reverse=True)
    tight = targets[-1]
    study = None
    if args.ws_blocks_study:  # the plain solver's error per sweep for several block counts (training head 999)
        t0 = time.time()
        cands = [int(v) for v in args.ws_blocks_study.split(",") if v.strip()]
        study = {"per_blocks": W.blocks_study(g, args.ws_test_n, 999, targets, args.ws_study_sweeps, cands,
                                              device=local, lanes=args.lanes), "study_s": time.time() - t0}
        log(f"blocks study: {study}")
    tuning = None
    if args.ws_tune_blocks:  # blocks per update picked on a training head (seed 999), then used throughout
        t0 = time.time()
        args.ws_blocks, trials = W.tune_blocks(g, args.ws_test_n, 999, args.ws_target, args.ws_max_sweeps,
                                               device=local, lanes=args.lanes)
        tuning = {"chosen": args.ws_blocks, "ms_to_target": {str(b): ms for b, ms in trials.items()},
                  "tuning_s": time.time() - t0}
        log(f"blocks per update: {tuning}")
    t0 = time.time()
    pairs = W.make_training_pairs(g, args.ws_pairs, args.ws_train_n, args.ws_train_sweeps, device=local, log=log,
                                  blocks=args.ws_blocks, lanes=args.lanes)
    t_data = time.time() - t0
    net = P.Net(g.nz, g.ny, g.nx, seed=7, device=local)
    t0 = time.time()
    hist = W.train(net, pairs, epochs=args.ws_epochs, lr=1e-3, log=log)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del pairs
    torch.cuda.empty_cache()
    results = []
    for k in range(args.ws_tests):
        wl = W.head_workload(g, args.ws_test_n, 5000 + k, n_blocks=args.ws_blocks)
        x_true = S.voxelize(wl.phantom(), g, ss=2)
        rec = S.make_histories_device(wl, device=f"cuda:{local}")
        ctx = P.Context(g, n_blocks=wl.n_blocks, device=local, lanes=args.lanes)
        r = {"seed": 5000 + k}
        for name, use in (("plain", None), ("warm", net)):
            ctx.load(rec)  # fresh: x = 0
            torch.cuda.synchronize()
            tw = time.perf_counter()
            ctx.block_weights()  # set-up, timed separately
            weights_s = time.perf_counter() - tw
            res = W.solve_to_target(ctx, x_true, g, tight, args.ws_max_sweeps, net=use)
            res["block_weights_seconds"] = weights_s
            res["seconds_to"] = {str(t): (lambda ms: None if ms is None else ms / 1e3)(W.ms_to_target(res, t))
                                 for t in targets}
            r[name] = res
            log(f"test {k} {name}: {res}")
        ctx.close()
        del rec
        torch.cuda.empty_cache()
        results.append(r)
    # the warm-started, batched form: several held-out heads of uneven size
    # advanced by one batch (graph branches; the batch forms every block weight
    # before the first timed sweep), plain against warm-started
    batched = None
    sizes = [int(float(v)) for v in args.ws_batch.split(",") if v.strip()] if args.ws_batch else []
    if sizes:
        wls = [W.head_workload(g, n, 6000 + k, n_blocks=args.ws_blocks) for k, n in enumerate(sizes)]
        truths = [S.voxelize(w.phantom(), g, ss=2) for w in wls]
        ctxs = []
        for w in wls:
            rec = S.make_histories_device(w, device=f"cuda:{local}")
            c = P.Context(g, n_blocks=w.n_blocks, device=local, lanes=args.lanes)
            c.load(rec)
            del rec
            torch.cuda.empty_cache()
            ctxs.append(c)
        zero = np.zeros(g.m, dtype=np.float32)
        batched = {"histories": sizes}
        with P.Batch(ctxs, mode=P.BATCH_GRAPH_BRANCHES) as b:
            for name, use in (("plain", None), ("warm", net)):
                for c in ctxs:
                    c.set_x0(zero)
                res = W.solve_batch_to_target(b, ctxs, truths, g, tight, args.ws_max_sweeps, net=use)
                res["seconds_to"] = {str(t): next((ms / 1e3 for e, ms in zip(res["worst_errors"], res["ms_at"])
                                                   if e <= t), None) for t in targets}
                batched[name] = res
                log(f"batch {name}: {res}")
        for c in ctxs:
            c.close()
        batched["speedup"] = {str(t): (batched["plain"]["seconds_to"][str(t)] / batched["warm"]["seconds_to"][str(t)]
                                       if batched["plain"]["seconds_to"][str(t)] and batched["warm"]["seconds_to"][str(t)]
                                       else None) for t in targets}
    net.close()

    def mean_s(name, t):
        v = [r[name]["seconds_to"][str(t)] for r in results]
        return statistics.mean(v) if v and all(x is not None for x in v) else None

    plain = {str(t): mean_s("plain", t) for t in targets}
    warm = {str(t): mean_s("warm", t) for t in targets}
    first = str(targets[0])
    return {
        "batched": batched,
        "metric": "time-to-image at <=1% mean RSP error", "unit": "s", "higher_is_better": False,
        "warm_seconds": warm[first], "plain_seconds": plain[first],
        "speedup": plain[first] / warm[first] if plain[first] and warm[first] else None,
        "by_target": {t: {"plain_seconds": plain[t], "warm_seconds": warm[t],
                          "speedup": plain[t] / warm[t] if plain[t] and warm[t] else None} for t in plain},
        "config": {"workload": f"warmstart_head200x200x48_{args.ws_test_n}", "grid": "200x200x48 @ 1x1x2 mm",
                   "test_histories": args.ws_test_n, "n_blocks": args.ws_blocks, "targets": targets,
                   "training_pairs": args.ws_pairs, "training_histories": args.ws_train_n,
                   "training_target": f"plain solver after {args.ws_train_sweeps} sweeps", "epochs": args.ws_epochs,
                   "lanes_per_history": args.lanes},
        "tests": results, "train_loss": hist, "training_data_s": t_data, "training_s": t_train,
        "blocks_tuning": tuning, "blocks_study": study,
    }


def run_warmstart(args):
    """The time-to-image leg alone (see time_to_image), as its own JSON line."""
    import torch

    from paper_1707_05014_gb300 import build as B

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    B.build()
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    tti = time_to_image(args, local, log)
    line = {"metric": tti["metric"], "value": tti["warm_seconds"], "unit": "s", "n_gpus": 1,
            "higher_is_better": False, "data": "synthetic", "dtype": "f32", "config": tti["config"],
            "plain_seconds": tti["plain_seconds"], "speedup": tti["speedup"],
            **{k: tti[k] for k in ("by_target", "tests", "train_loss", "training_data_s", "training_s",
                                   "blocks_tuning", "blocks_study", "batched")}}
    print(json.dumps(line), flush=True)
    return 0


def run_table2(args):
    """Table 2 style accuracy study on the synthetic insert phantom: DROP and
    CARP (both with TVS, as in Sec. 4.2), ROI mean / std / %error per insert."""
    import numpy as np
    import torch

    from paper_1707_05014_gb300 import build as B
    from paper_1707_05014_gb300 import pct as P
    from paper_1707_05014_gb300 import synthetic as S

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    B.build()
    g = S.Grid(160, 160, 32, 1.25, 1.25, 1.25)
    wl = S.Workload(f"catphan_{args.t2_n}", g, args.t2_n, 404, 0, g.radius, 18.0, args.t2_blocks, args.t2_sweeps,
                    "catphan")
    rec = S.make_histories_device(wl, device=f"cuda:{local}")
    out = {}
    for name, flags in (("DROP", 0), ("CARP", P.FLAG_CARP)):
        with P.Context(g, n_blocks=wl.n_blocks, flags=flags, tvs_beta0=args.t2_tvs, carp_strings=args.t2_strings,
                       device=local) as ctx:
            ctx.load(rec)
            if args.hull:
                ctx.carve_hull(args.hull_wepl, args.hull_dilate)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            st = torch.cuda.current_stream()
            e0.record(st)
            ctx.iterate(wl.n_sweeps)
            e1.record(st)
            x = ctx.get_rsp().astype(np.float64)
            out[name] = {"rows": S.roi_stats(x, g), "seconds": e0.elapsed_time(e1) / 1e3}
    line = {"metric": "ROI RSP accuracy (Table 2 format)", "unit": "RSP", "data": "synthetic",
            "config": {"workload": wl.name, "grid": "160x160x32 @ 1.25 mm", "histories": wl.n, "blocks": wl.n_blocks,
                       "carp_strings": args.t2_strings,
                       "hull": (f"carved: WEPL <= {args.hull_wepl} mm, dilate {args.hull_dilate}") if args.hull else "none",
                       "iterations": wl.n_sweeps, "tvs_beta0": args.t2_tvs,
                       "phantom": "150 mm RSP-1.0 cylinder, seven 12 mm inserts at Table 2's true RSPs"},
            "results": out}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1707_05014_gb300 import build as B
    from paper_1707_05014_gb300 import pct as P
    from paper_1707_05014_gb300 import synthetic as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    wl = main_workload(args, rank)  # weak scaling: each rank its own reconstruction
    g = wl.grid
    rec = S.make_histories_device(wl, device=f"cuda:{local}")
    torch.cuda.synchronize()

    flags = P.FLAG_PROFILE | (P.FLAG_NO_SORT if args.no_sort else 0)
    ctx = P.Context(g, n_blocks=wl.n_blocks, flags=flags, node_step=args.node_step, device=local, lanes=args.lanes)
    ctx.load(rec, borrow=True)
    hull = None
    if args.hull:  # object hull carved from the data (untimed set-up, like the load)
        ctx.carve_hull(args.hull_wepl, args.hull_dilate)
        hull = ctx.get_hull()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctx.iterate(1)
        ctx.last_sweep_times()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ctx.launches
    fused_ms = []
    apply_ms = []
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.iterate(1)
        f, a = ctx.last_sweep_times()  # waits for the sweep; reads its per-kernel events
        fused_ms.extend(f.tolist())
        apply_ms.extend(a.tolist())
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = ctx.launches - launches0
    ms = max_over_ranks(ms, device=f"cuda:{local}")
    value = wl.n * args.steps * world / (ms / 1e3)

    # roofline of the dominant kernel (fused MLP + projection): ALU-bound
    peaks, src = _peaks()
    per_block = wl.n / wl.n_blocks
    avg_fused_s = statistics.mean(fused_ms) / 1e3
    ctx_rows = P.Context(g, n_blocks=1, node_step=args.node_step, device=local)  # runs per history (unit count)
    sample = {k: v[: min(wl.n, 200_000)] for k, v in rec.items()}
    ctx_rows.load(sample, borrow=True)
    if hull is not None:
        ctx_rows.set_hull(hull)
    rp = ctx_rows.rows(0, len(sample["t0"]))[0]
    runs_per_history = float(rp[-1].item()) / len(sample["t0"])
    ctx_rows.close()
    ops_per_history = OPS_PER_MLP_NODE * (ctx.K + 1) + OPS_PER_RUN * runs_per_history
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = ALU_LANES_PER_SM * N_SMS * sm_mhz * 1e6 / 1e12  # Tops/s
    achieved = ops_per_history * per_block / avg_fused_s / 1e12
    traffic = traffic_per_launch(ncu_counters(), args, per_block)
    hbm_achieved = 44.0 * per_block / avg_fused_s / 1e9
    # the library's own roof microbenchmarks: L2 atomics, L2 gathers, ALU issue
    mr = P.measure_roofs(local)
    per_s = per_block / avg_fused_s
    measured = {
        "l2_atomic": {"achieved": runs_per_history * per_s, "peak": mr["l2_red_per_s"], "unit": "atomics/s",
                      "peak_coherent_lines": mr["l2_red_coherent_per_s"]},
        "l2_gather": {"achieved": runs_per_history * per_s, "peak": mr["l2_gather_per_s"], "unit": "loads/s"},
        "alu_issue": {"achieved": ops_per_history * per_s, "peak": mr["alu_ops_per_s"], "unit": "ops/s",
                      "fma_chain_peak": mr["fma_ops_per_s"]},
        "source": (f"pct_measure_roofs: random float atomics / 4 B gathers in an {mr['array_bytes'] >> 20} MB "
                   f"array (L2 {mr['l2_bytes'] >> 20} MB), integer and FMA chains; {mr['sms']} SMs"),
    }
    for k in ("l2_atomic", "l2_gather", "alu_issue"):
        measured[k]["frac"] = measured[k]["achieved"] / measured[k]["peak"]
    kname = "drop_fused_hull_kernel" if args.hull else ("drop_group_kernel" if args.lanes > 1 else "drop_fused_kernel")
    roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
            "frac": achieved / alu_peak, "traffic": traffic,
            "peak_source": f"{ALU_LANES_PER_SM} lanes x {N_SMS} SMs x {sm_mhz:.0f} MHz",
            "ops_per_history": ops_per_history, "runs_per_history": runs_per_history, "mlp_nodes": ctx.K + 1,
            "avg_launch_ms": avg_fused_s * 1e3, "histories_per_launch": per_block,
            "fused_share_of_step": sum(fused_ms) / ms,
            "hbm": {"achieved": hbm_achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": hbm_achieved / peaks["hbm_gbs"], "peak_source": src, "algorithmic_bytes": "44 B/history"},
            "measured_roofs": measured}

    # end to end through the public API from pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        host = {}
        for k, v in rec.items():  # pinned host copies, one field at a time
            host[k] = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
            host[k].copy_(v)
        del rec
        torch.cuda.empty_cache()
        ctx.close()
        ctx2 = P.Context(g, n_blocks=wl.n_blocks, node_step=args.node_step, device=local, lanes=args.lanes)
        xs = []
        times = []
        loads = []
        for i in range(1 + args.e2e_steps):
            barrier()
            t0 = time.perf_counter()
            ctx2.load(host)  # returns once the records are validated (it synchronises)
            tl = time.perf_counter()
            if args.hull:
                ctx2.carve_hull(args.hull_wepl, args.hull_dilate)
            ctx2.iterate(args.e2e_sweeps)
            xs.append(ctx2.get_rsp())
            dt = time.perf_counter() - t0
            if i > 0:
                times.append(dt)
                loads.append(tl - t0)
        ctx2.close()
        e2e_val = wl.n * args.e2e_sweeps * world / statistics.mean(times)
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 44 * wl.n,
               "d2h_bytes_per_step": 4 * g.m, "sweeps_per_step": args.e2e_sweeps,
               "includes": "H2D copy, validation, block counts, " + ("hull carving, " if args.hull else "") +
                           "sweeps, D2H of x",
               "seconds_per_step": statistics.mean(times), "load_seconds": statistics.mean(loads),
               "sweeps_and_readback_seconds": statistics.mean(times) - statistics.mean(loads)}
    else:
        ctx.close()

    tti = None
    if rank == 0 and args.time_to_image:
        # second half of the metric: time to <= 1 % mean RSP error, warm start
        # against the plain solver, the network trained in this run
        host = rec = None  # the throughput leg's records (host and device) are no longer needed
        torch.cuda.empty_cache()
        log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
        full = time_to_image(args, local, log)
        tti = {k: full[k] for k in ("metric", "unit", "higher_is_better", "warm_seconds", "plain_seconds", "speedup",
                                    "by_target", "config", "training_data_s", "training_s", "blocks_tuning",
                                    "blocks_study")}
        tti["tests"] = [{"seed": r["seed"], **{m: {"seconds_to": r[m]["seconds_to"], "sweeps": r[m]["sweeps"],
                                                   "errors": r[m]["errors"],
                                                   "block_weights_seconds": r[m]["block_weights_seconds"],
                                                   **({"net_used": r[m]["net_used"]} if m == "warm" else {})}
                                               for m in ("plain", "warm")}} for r in full["tests"]]
        bt = full["batched"]
        tti["batched"] = None if bt is None else {
            "histories": bt["histories"], "speedup": bt["speedup"],
            **{m: {"seconds_to": bt[m]["seconds_to"], "sweeps": bt[m]["sweeps"], "errors": bt[m]["errors"],
                   "net_used": bt[m]["net_used"]} for m in ("plain", "warm")}}

    cpu = None
    if rank == 0 and args.cpu_sample > 0:
        crec = oracle_sample(wl, args.cpu_sample)
        r1, dt1, _ = oracle_rate(wl, crec, node_step=args.node_step, threads=1)
        r, dt, cores = oracle_rate(wl, crec, node_step=args.node_step, threads=0)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample} histories of the same workload, 1 sweep, {wl.n_blocks} blocks "
                         f"(FP64 oracle, each block's histories split over {cores} OpenMP threads, {dt:.1f} s; "
                         f"single thread {dt1:.1f} s)",
               "single_thread_value": r1}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name + ("_hull" if args.hull else "") + (f"_step{args.node_step:g}mm" if args.node_step > 0 else ""),
                       "grid": grid_text(g),
                       "mlp_node_step_mm": args.node_step if args.node_step > 0 else min(g.hx, g.hy, g.hz) / 2,
                       "lanes_per_history": args.lanes,
                       "histories_per_gpu": wl.n, "angles": wl.n_angles or "continuous", "n_blocks": wl.n_blocks,
                       "step": "one DROP sweep over all histories", "parallelism": f"replicas{world}",
                       "l2": f"records {44 * wl.n / 1e9:.1f} GB per sweep > 129 MB L2 (no flush needed); x and delta L2-resident",
                       "hull": (f"carved from the data: rows of histories with WEPL <= {args.hull_wepl} mm are air, "
                                f"hull dilated by {args.hull_dilate} voxel") if args.hull else "none (MLP between the planes)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "time_to_image": tti, "gpu_launches": launches,
            "clocks": clk,
            "host_threads": _cpu_threads(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None, help="histories per GPU (default: the workload's own)")
    ap.add_argument("--blocks", type=int, default=0,
                    help="DROP blocks of the throughput workload (default: the workload's own; a profile of one "
                         "full-size launch uses --n 20000000 --blocks 1)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--e2e-sweeps", type=int, default=10)
    ap.add_argument("--cpu-sample", type=int, default=1_000_000)
    ap.add_argument("--ref-sample", type=int, default=1_000_000)
    ap.add_argument("--lanes", type=int, default=1, help="lanes per history in the fused kernel (1, 2, 4, 8, 16, 32)")
    ap.add_argument("--no-sort", action="store_true", help="keep each block in load order (A/B of the ordering)")
    ap.add_argument("--hull", action="store_true", help="head / table2: MLP inside a hull carved from the data")
    ap.add_argument("--node-step", type=float, default=0.0, help="head: MLP node spacing in mm (default min(h)/2)")
    ap.add_argument("--hull-wepl", type=float, default=1.0, help="carving: histories with WEPL <= this (mm) are air")
    ap.add_argument("--hull-dilate", type=int, default=1, help="carving: 6-neighbour growth steps of the hull")
    ap.add_argument("--workload", default="head200",
                    choices=["head200", "head", "tiny", "batched", "precision", "warmstart", "table2"])
    ap.add_argument("--t2-n", type=int, default=200_000_000)
    ap.add_argument("--t2-blocks", type=int, default=600, help="DROP blocks; CARP: blocks split over the strings")
    ap.add_argument("--t2-strings", type=int, default=60)
    ap.add_argument("--t2-sweeps", type=int, default=10)
    ap.add_argument("--t2-tvs", type=float, default=0.02)
    ap.add_argument("--no-time-to-image", dest="time_to_image", action="store_false",
                    help="skip the time-to-image leg of the default run")
    ap.add_argument("--ws-pairs", type=int, default=200)
    ap.add_argument("--ws-train-n", type=int, default=50_000_000)
    ap.add_argument("--ws-train-sweeps", type=int, default=3)
    ap.add_argument("--ws-blocks", type=int, default=50)
    ap.add_argument("--ws-tune-blocks", action="store_true",
                    help="time to image: tune the block count for the plain solver's time to --ws-target on a "
                         "training head and use it for both solvers (default: --ws-blocks)")
    ap.add_argument("--ws-blocks-study", default="20,50,100,200",
                    help="block counts of the plain-solver study reported beside the time to image ('' to skip)")
    ap.add_argument("--ws-study-sweeps", type=int, default=4)
    ap.add_argument("--ws-epochs", type=int, default=10)
    ap.add_argument("--ws-tests", type=int, default=2)
    ap.add_argument("--ws-test-n", type=int, default=1_000_000_000)
    ap.add_argument("--ws-target", type=float, default=0.01)
    ap.add_argument("--ws-target2", type=float, default=0.006, help="a tighter second target (<= 0: none)")
    ap.add_argument("--ws-max-sweeps", type=int, default=6)
    ap.add_argument("--ws-batch", default="1e9,5e8,2.5e8",
                    help="histories of the held-out heads solved together as one batch ('' to skip)")
    ap.add_argument("--n-recon", type=int, default=32, help="reconstructions of the batched workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "table2":
        return run_table2(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
