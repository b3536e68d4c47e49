"""A DROP block shared by several ranks (Sec. 1 / Sec. 3.1: the histories are
distributed over processors), emulated on one GPU: two contexts hold the two
halves of every block; each block update is pct_block_partial on both, a
device-side sum of their update buffers and run counts (what an all-reduce
gives each rank), then pct_block_apply with the sums on both. Both ranks then
hold the oracle's DROP image of the whole set."""
import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

RSP_TOL = 1e-3


@pytest.fixture(scope="module")
def pct():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1707_05014_gb300 import build, pct as P

    build.build()
    return P


def _shares(n_blocks, ranks, per_rank_block):
    """History indices of each rank: rank r takes every ranks-th history of each
    global block b = [b n/B, (b+1) n/B), so that its own block b (its histories
    [b m, (b+1) m)) is its share of global block b."""
    per_block = ranks * per_rank_block
    return [np.concatenate([np.arange(b * per_block + r, (b + 1) * per_block, ranks) for b in range(n_blocks)])
            for r in range(ranks)]


@pytest.mark.parametrize("kind,B,m,lam,flags", [("water", 5, 4000, 1.0, 0), ("head", 4, 10_000, 1.5, 1)],
                         ids=["water", "head_clamp"])
def test_two_ranks_sharing_every_block_equal_the_oracle(pct, oracle, kind, B, m, lam, flags):
    import torch

    G, sweeps = 2, 2
    n = B * G * m
    wl = S.tiny_workload(n, seed=91) if kind == "water" else S.head_workload(n, seed=92)
    g = wl.grid
    rec = S.make_histories(wl)
    clamp_min = 0.005 if flags & pct.FLAG_CLAMP else 0.0
    ctxs = []
    for idx in _shares(B, G, m):
        c = pct.Context(g, n_blocks=B, lam=lam, flags=flags, clamp_min=clamp_min)
        c.load(S.subset(rec, idx))
        ctxs.append(c)
    dev = torch.device("cuda")
    delta = [torch.empty(g.m, dtype=torch.float32, device=dev) for _ in range(G)]
    counts = [torch.empty(g.m, dtype=torch.float32, device=dev) for _ in range(G)]
    count_sums = []
    for sweep in range(sweeps):
        for b in range(B):
            for r, c in enumerate(ctxs):
                c.block_partial(b, delta[r], counts[r] if sweep == 0 else None)
            dsum = delta[0] + delta[1]
            if sweep == 0:  # the run counts of a block are reduced once and kept
                count_sums.append(counts[0] + counts[1])
            for c in ctxs:
                c.block_apply(dsum, count_sums[b])
    xs = [c.get_rsp().astype(np.float64) for c in ctxs]
    for c in ctxs:
        c.close()
    assert np.array_equal(xs[0], xs[1])  # every rank applies the same sums to the same x
    xo = oracle.drop(g, rec, B, sweeps, lam=lam, mode=oracle.MODE_FP32,
                     clamp_min=clamp_min if flags & pct.FLAG_CLAMP else None)
    err = np.abs(xs[0] - xo) / np.maximum(np.abs(xo), 1.0)
    assert err.max() <= RSP_TOL, err.max()
    # the summed counts are the global block's run counts
    for b in range(B):
        assert np.array_equal(count_sums[b].cpu().numpy().astype(np.float64),
                              oracle.block_counts(g, rec, B, b, mode=oracle.MODE_FP32))


def test_partial_leaves_x_and_apply_needs_both_buffers(pct):
    import torch

    wl = S.tiny_workload(3000, seed=93)
    with pct.Context(wl.grid, n_blocks=2) as c:
        c.load(S.make_histories(wl))
        d = torch.empty(wl.grid.m, dtype=torch.float32, device="cuda")
        c.block_partial(1, d)
        assert float(np.abs(c.get_rsp()).max()) == 0.0  # x is untouched by the partial
        assert float(d.abs().max()) > 0.0
        with pytest.raises(pct.PctError) as ei:
            c.block_partial(2, d)
        assert ei.value.code == -1
