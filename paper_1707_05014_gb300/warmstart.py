"""Warm-started reconstruction: plain DROP sweeps plus the learned initial image.

Solve (every step runs in the library's kernels; this module only sequences
the calls):
  1. one DROP sweep from x = 0 gives x1 (Sec. 2.1, Fig. 1);
  2. the network gives x0' = x1 + f(x1);
  3. fallback: if the data residual |b - A x0'|^2 (on a 1/64 sample of the
     histories) is larger than that of x1, keep x1 (the plain solver's data
     fit decides);
  4. further DROP sweeps from the chosen image.

Training pairs are (x1, x_S): the first sweep and the plain solver's result
after S sweeps, from seeded random head phantoms (synthetic.py). The network
learns to jump from the first sweep towards the plain solver's answer.
"""
from __future__ import annotations

import time
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import pct as P
from . import synthetic as S


def training_grid() -> S.Grid:
    """200 x 200 x 48 voxels of 1 x 1 x 2 mm (1.92M voxels)."""
    return S.Grid(200, 200, 48, 1.0, 1.0, 2.0)


def head_workload(grid: S.Grid, n: int, seed: int, n_blocks: int = 10) -> S.Workload:
    """Seeded random head (outer semi-axes and inserts jittered by +-15 %), the
    recipe of synthetic.head200_workload on `grid`."""
    return S.Workload(f"warm_head{seed}_{n}", grid, n, seed, 90, grid.radius,
                      min(46.0, 0.5 * grid.nz * grid.hz - 2.0), n_blocks, 10, "head", 0.15)


def plain_pair(wl: S.Workload, sweeps: int, device: int = 0, lam: float = 1.0, lanes: int = 1):
    """(x1, x_sweeps) of one plain-solver reconstruction, as CUDA tensors."""
    import torch

    rec = S.make_histories_device(wl, device=f"cuda:{device}")
    with P.Context(wl.grid, n_blocks=wl.n_blocks, lam=lam, device=device, lanes=lanes) as ctx:
        ctx.load(rec)
        del rec
        ctx.iterate(1)
        x1 = ctx.get_rsp(device=True)
        ctx.iterate(sweeps - 1)
        xs = ctx.get_rsp(device=True)
        torch.cuda.synchronize()
    return x1, xs


def make_training_pairs(grid: S.Grid, n_pairs: int, n_histories: int, sweeps: int, seed0: int = 1000,
                        device: int = 0, log: Optional[Callable[[str], None]] = None, blocks: int = 10,
                        lanes: int = 1):
    pairs = []
    t0 = time.time()
    for k in range(n_pairs):
        pairs.append(plain_pair(head_workload(grid, n_histories, seed0 + k, n_blocks=blocks), sweeps, device,
                                lanes=lanes))
        if log and (k + 1) % 25 == 0:
            log(f"training pairs {k + 1}/{n_pairs} ({time.time() - t0:.0f} s)")
    return pairs


def train(net: P.Net, pairs: Sequence[Tuple], epochs: int, lr: float = 1e-3, seed: int = 0,
          log: Optional[Callable[[str], None]] = None) -> List[float]:
    """Adam on the L1 loss, one pair per step, shuffled every epoch; returns the
    mean loss of each epoch."""
    rng = np.random.Generator(np.random.Philox(seed))
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(pairs))
        losses = []
        for i, k in enumerate(order):
            x1, xs = pairs[k]
            want = i % 8 == 0
            l = net.train_step(x1, xs, lr=lr * (0.5 ** (ep // max(1, epochs // 3))), want_loss=want)
            if want:
                losses.append(l)
        hist.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep + 1}/{epochs}: L1 {hist[-1]:.5f}")
    return hist


def solve_to_target(ctx: P.Context, x_true: np.ndarray, grid: S.Grid, target: float, max_sweeps: int,
                    net: Optional[P.Net] = None, check_stride: int = 64) -> Dict:
    """Sweeps until the mean RSP error (interior ROI) is <= target. Times only
    the GPU work (sweeps, network, residual check) with CUDA events; the error
    evaluation against the known phantom is outside the timed region. If the
    block weights are not formed yet (ctx.block_weights), the first sweep
    forms them inside the timed region."""
    import torch

    stream = torch.cuda.current_stream()
    t_ms = 0.0
    errs = []
    used_net = False

    def timed(fn):
        nonlocal t_ms
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t_ms += e0.elapsed_time(e1)
        return out

    def err():
        return S.mean_rsp_error(ctx.get_rsp().astype(np.float64), x_true, grid)

    ms_at = []  # GPU time spent when each error was reached
    sweeps = 0
    timed(lambda: ctx.iterate(1))
    sweeps = 1
    if net is not None:
        used_net = timed(lambda: warm_start(ctx, net, check_stride))
    errs.append(err())
    ms_at.append(t_ms)
    while errs[-1] > target and sweeps < max_sweeps:
        timed(lambda: ctx.iterate(1))
        sweeps += 1
        errs.append(err())
        ms_at.append(t_ms)
    return {"reached": errs[-1] <= target, "sweeps": sweeps, "ms": t_ms, "errors": errs, "ms_at": ms_at,
            "net_used": used_net}


def ms_to_target(result: Dict, target: float) -> Optional[float]:
    """GPU time (ms) at which a solve_to_target result first reached `target`
    (None if it never did)."""
    return next((ms for e, ms in zip(result["errors"], result["ms_at"]) if e <= target), None)


def warm_start(ctx: P.Context, net: P.Net, check_stride: int = 64) -> bool:
    """Steps 2-3 of the solve on one context after its first sweep: x0 = x1 +
    f(x1), kept only if its data residual on every check_stride-th history is
    not larger than that of x1. Returns whether the network's image is kept."""
    x1 = ctx.get_rsp(device=True)
    r1 = ctx.residual(check_stride)
    ctx.set_x0(net.forward(x1))
    r0 = ctx.residual(check_stride)
    if r0 > r1:  # fallback: the plain solver's image is better
        ctx.set_x0(x1)
        return False
    return True


def solve_batch_to_target(batch: P.Batch, ctxs: Sequence[P.Context], x_trues: Sequence[np.ndarray],
                          grid: S.Grid, target: float, max_sweeps: int, net: Optional[P.Net] = None,
                          check_stride: int = 64) -> Dict:
    """solve_to_target for several reconstructions advanced together by one
    batch (pct_batch_iterate): every sweep is one batched call over all of
    them; with a network, each reconstruction is warm-started (with its own
    residual fallback) after the first sweep. Sweeps continue until every
    reconstruction's mean RSP error is <= target. Times the GPU work with CUDA
    events; the error evaluation is outside the timed region."""
    import torch

    stream = torch.cuda.current_stream()
    t_ms = 0.0

    def timed(fn):
        nonlocal t_ms
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t_ms += e0.elapsed_time(e1)
        return out

    def errs_now():
        return [S.mean_rsp_error(c.get_rsp().astype(np.float64), xt, grid) for c, xt in zip(ctxs, x_trues)]

    def sweep():
        batch.iterate(1)
        batch.sync()

    timed(sweep)
    sweeps = 1
    used = [False] * len(ctxs)
    if net is not None:
        used = timed(lambda: [warm_start(c, net, check_stride) for c in ctxs])
    errs = [errs_now()]
    ms_at = [t_ms]
    while max(errs[-1]) > target and sweeps < max_sweeps:
        timed(sweep)
        sweeps += 1
        errs.append(errs_now())
        ms_at.append(t_ms)
    per = [next((k + 1 for k, e in enumerate(errs) if e[r] <= target), None) for r in range(len(ctxs))]
    return {"reached": max(errs[-1]) <= target, "sweeps": sweeps, "ms": t_ms, "sweeps_to_target": per,
            "errors": [[e[r] for e in errs] for r in range(len(ctxs))], "ms_at": ms_at,
            "worst_errors": [max(e) for e in errs], "net_used": used}


def pick_blocks(trial: Callable[[int, Optional[float]], Optional[float]], candidates: Sequence[int]) -> Tuple[int, Dict]:
    """Blocks-per-update autotuner: the DROP block count B (Sec. 2.1 leaves it
    to the user) with the shortest time to the target.

    trial(B, limit_ms) returns the time (ms) one reconstruction with B blocks
    takes to reach the target, or None if it does not reach it; limit_ms is
    the best time so far (None at first), which a trial may use to give up
    early. Candidates are tried in the given order. Returns the chosen B and
    every candidate's result; raises ValueError if none reaches the target.
    B changes the iteration itself, so it is tuned for time to a result,
    never for throughput."""
    if not candidates:
        raise ValueError("no block counts to try")
    results: Dict[int, Optional[float]] = {}
    best_b, best_ms = None, None
    for b in candidates:
        if b < 1:
            raise ValueError(f"block count {b} < 1")
        ms = trial(b, best_ms)
        results[b] = ms
        if ms is not None and (best_ms is None or ms < best_ms):
            best_b, best_ms = b, ms
    if best_b is None:
        raise ValueError("no block count reached the target")
    return best_b, results


def blocks_study(grid: S.Grid, n: int, seed: int, targets: Sequence[float], sweeps: int,
                 candidates: Sequence[int] = (20, 50, 100, 200), device: int = 0, lanes: int = 1) -> Dict:
    """The plain solver on one seeded training head for every block count B:
    the mean RSP error after each of `sweeps` sweeps and the GPU time at which
    each target was first reached (None if not within the sweeps). Shows the
    trade-off the block count sets: more blocks converge faster per sweep, and
    with noisy data stall higher (the error can grow again over later
    sweeps)."""
    import torch

    out = {}
    for b in candidates:
        wl = head_workload(grid, n, seed, n_blocks=b)
        x_true = S.voxelize(wl.phantom(), grid, ss=2)
        rec = S.make_histories_device(wl, device=f"cuda:{device}")
        with P.Context(grid, n_blocks=b, device=device, lanes=lanes) as ctx:
            ctx.load(rec)
            del rec
            torch.cuda.empty_cache()
            ctx.block_weights()  # set-up, outside the timed sweeps
            r = solve_to_target(ctx, x_true, grid, -1.0, sweeps)  # every sweep (no target stops it)
        out[str(b)] = {"errors": r["errors"], "ms_at": r["ms_at"],
                       "seconds_to": {str(t): (lambda ms: None if ms is None else ms / 1e3)(ms_to_target(r, t))
                                      for t in targets}}
    return out


def tune_blocks(grid: S.Grid, n: int, seed: int, target: float, max_sweeps: int,
                candidates: Sequence[int] = (20, 50, 100, 200), device: int = 0, lanes: int = 1) -> Tuple[int, Dict]:
    """pick_blocks on one seeded training head: for each B, a plain
    reconstruction from x = 0 timed to the target mean RSP error (the known
    phantom of a training case decides; held-out cases are never used)."""
    import torch

    def trial(b: int, limit_ms: Optional[float]) -> Optional[float]:
        wl = head_workload(grid, n, seed, n_blocks=b)
        x_true = S.voxelize(wl.phantom(), grid, ss=2)
        rec = S.make_histories_device(wl, device=f"cuda:{device}")
        with P.Context(grid, n_blocks=b, device=device, lanes=lanes) as ctx:
            ctx.load(rec)
            del rec
            torch.cuda.empty_cache()
            ctx.block_weights()  # set-up, outside the timed sweeps
            r = solve_to_target(ctx, x_true, grid, target, max_sweeps)
        return r["ms"] if r["reached"] else None

    return pick_blocks(trial, candidates)
