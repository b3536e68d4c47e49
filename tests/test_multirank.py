"""Multi-rank paths on CPU with the gloo backend (world size 2).

* bench.py's job time is the slowest rank's time (all-reduce MAX).
* The sharded-block design for several GPUs: the histories of every DROP block
  are split over the ranks; each rank sums its partial update delta and its
  partial run counts s_j, one all-reduce(sum) per block combines them, and
  every rank applies the same x update. The result must equal the single-rank
  DROP of the oracle (Sec. 2.1) -- checked here with the oracle's rows.
* CARP in the paper's distributed form (Sec. 2.2): strings spread over the
  ranks, one all-reduce(sum) of (touch * x_s, touch) per iteration; equal to
  the oracle's single-process CARP.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _max_worker(rank, world, port, out):
    import bench

    _init(rank, world, port)
    try:
        out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank)
    finally:
        dist.destroy_process_group()


def test_job_time_is_max_over_ranks():
    port = _port()
    out = mp.Manager().dict()
    mp.spawn(_max_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == 15.0


def _shard_worker(rank, world, port, out):
    import oracle as O
    from paper_1707_05014_gb300 import synthetic as S

    _init(rank, world, port)
    try:
        wl = S.tiny_workload(3000, seed=81)
        g = wl.grid
        rec = S.make_histories(wl)
        B, sweeps, lam = 3, 2, 1.0
        rp, vox, ln = O.rows(g, rec)
        x = np.zeros(g.m)
        for _ in range(sweeps):
            for b in range(B):
                lo, hi = b * 3000 // B, (b + 1) * 3000 // B
                mine = range(lo + rank, hi, world)  # this rank's share of the block
                delta = np.zeros(g.m)
                cnt = np.zeros(g.m)
                for i in mine:
                    j, l = vox[rp[i]:rp[i + 1]], ln[rp[i]:rp[i + 1]]
                    nn = float((l * l).sum())
                    if nn <= 0:
                        continue
                    r = lam * (float(rec["wepl"][i]) - float((l * x[j]).sum())) / nn
                    np.add.at(delta, j, l * r)
                    np.add.at(cnt, j, 1.0)
                t = torch.from_numpy(np.stack([delta, cnt]))
                dist.all_reduce(t)  # the one exchange per block
                d, c = t[0].numpy(), t[1].numpy()
                x = x + np.where(c > 0, d / np.maximum(c, 1.0), 0.0)
        out[rank] = x
    finally:
        dist.destroy_process_group()


def test_sharded_blocks_equal_single_rank_drop(oracle):
    from paper_1707_05014_gb300 import synthetic as S

    port = _port()
    out = mp.Manager().dict()
    mp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
    wl = S.tiny_workload(3000, seed=81)
    ref = oracle.drop(wl.grid, S.make_histories(wl), 3, 2, mode=oracle.MODE_FP32)
    for r in (0, 1):
        assert np.abs(out[r] - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
    assert np.array_equal(out[0], out[1])


def _carp_worker(rank, world, port, out):
    import oracle as O
    from paper_1707_05014_gb300 import synthetic as S

    _init(rank, world, port)
    try:
        wl = S.tiny_workload(3000, seed=82)
        g = wl.grid
        rec = S.make_histories(wl)
        n, B, S_, sweeps = 3000, 6, 3, 2  # strings of two blocks of 500 histories
        per = B // S_
        x = np.zeros(g.m)
        for _ in range(sweeps):
            num = np.zeros(g.m)
            den = np.zeros(g.m)
            for s in range(rank, S_, world):  # this rank's strings (the paper's one string per processor)
                lo, hi = s * per * n // B, (s + 1) * per * n // B
                sub = S.subset(rec, slice(lo, hi))
                xs = O.drop(g, sub, per, 1, x0=x)  # the string's DROP sweep from the common x
                touch = np.zeros(g.m)
                touch[np.unique(O.rows(g, sub)[1])] = 1.0
                num += touch * xs
                den += touch
            t = torch.from_numpy(np.stack([num, den]))
            dist.all_reduce(t)  # the one exchange per iteration
            num, den = t[0].numpy(), t[1].numpy()
            x = np.where(den > 0, num / np.maximum(den, 1.0), x)
        out[rank] = x
    finally:
        dist.destroy_process_group()


def test_strings_on_ranks_equal_single_rank_carp(oracle):
    # CARP in the paper's distributed form (Sec. 2.2): the strings are spread
    # over the ranks, each sweeps its strings from the common image, and one
    # all-reduce(sum) of (touch * x_s, touch) per iteration forms the component
    # average. It must equal the oracle's single-process CARP.
    from paper_1707_05014_gb300 import synthetic as S

    port = _port()
    out = mp.Manager().dict()
    mp.spawn(_carp_worker, args=(2, port, out), nprocs=2, join=True)
    wl = S.tiny_workload(3000, seed=82)
    ref = oracle.carp(wl.grid, S.make_histories(wl), 3, 2, n_blocks=6, mode=oracle.MODE_FP32)
    for r in (0, 1):
        assert np.abs(out[r] - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
    assert np.array_equal(out[0], out[1])
