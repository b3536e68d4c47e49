"""The learned warm start gains over the plain solver: trained on plain-solver
reconstructions of seeded random heads, the network's x0 = x1 + f(x1) after one
sweep is closer to the true image than the plain solver after the same work,
and the warm-started solve stays ahead of the plain solver at every sweep
(about one sweep saved at this scale). Small scale (64 x 64 x 32 grid, 32
training pairs, 120 epochs: at 40 epochs the gain varied from run to run, the
training data coming from float-atomic reconstructions) so it runs in a
minute or two."""
import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1707_05014_gb300 import build, pct, warmstart

    build.build()
    return pct, warmstart


GRID = S.Grid(64, 64, 32, 3.125, 3.125, 3.125)
N_HIST, SWEEPS = 3_000_000, 8


@pytest.fixture(scope="module")
def trained(mods):
    P, W = mods
    pairs = W.make_training_pairs(GRID, 32, N_HIST, SWEEPS, seed0=500)
    net = P.Net(GRID.nz, GRID.ny, GRID.nx, seed=1)
    hist = W.train(net, pairs, epochs=120, lr=2e-3)
    yield net, hist
    net.close()


def test_warm_start_beats_plain_solver(mods, trained):
    P, W = mods
    g = GRID
    n, sweeps = N_HIST, SWEEPS
    net, hist = trained
    assert hist[-1] < hist[0]
    gains = []
    for seed in (900, 901):
        wl = W.head_workload(g, n, seed)
        x_true = S.voxelize(wl.phantom(), g, ss=2)
        rec = S.make_histories(wl)
        res = {}
        for name, use in (("plain", None), ("warm", net)):
            with P.Context(g, n_blocks=wl.n_blocks) as ctx:
                ctx.load(rec)
                res[name] = W.solve_to_target(ctx, x_true, g, 0.0, sweeps, net=use)
        plain, warm = res["plain"]["errors"], res["warm"]["errors"]
        print(seed, "plain", np.round(plain, 4), "warm", np.round(warm, 4), res["warm"]["net_used"])
        # the warm-started solve stays ahead of the plain solver sweep by
        # sweep, and its first image is about as good as two plain sweeps
        assert all(w < p for w, p in zip(warm[:4], plain[:4]))
        assert warm[0] <= 1.15 * plain[1]
        gains.append((plain[:4], warm[:4]))
    print("warm-start gains:", gains)


def test_batched_warm_start_reaches_the_target_in_fewer_sweeps(mods, trained):
    """Several reconstructions of uneven size advanced by one batch: with the
    network (each with its own residual fallback) every one stays ahead of the
    plain batch over the first three sweeps, and the batch reaches the plain batch's
    three-sweep errors in fewer sweeps in all. The saving is about one sweep
    for the 3M and 1.5M-history reconstructions and about two thirds of a
    sweep for the 800k-history one (noisier than the 3M-history training
    images), so a whole sweep is not asked of each."""
    P, W = mods
    net, _ = trained
    g = GRID
    wls = [W.head_workload(g, n, seed) for n, seed in ((3_000_000, 910), (1_500_000, 911), (800_000, 912))]
    recs = [S.make_histories(w) for w in wls]
    truths = [S.voxelize(w.phantom(), g, ss=2) for w in wls]
    runs = {}
    for name, use in (("plain", None), ("warm", net)):
        ctxs = []
        for w, r in zip(wls, recs):
            c = P.Context(g, n_blocks=w.n_blocks)
            c.load(r)
            ctxs.append(c)
        with P.Batch(ctxs, mode=P.BATCH_GRAPH_BRANCHES) as b:
            runs[name] = W.solve_batch_to_target(b, ctxs, truths, g, 0.0, 4, net=use)
        for c in ctxs:
            c.close()
    plain, warm = runs["plain"], runs["warm"]
    print("plain", np.round(plain["errors"], 4), "warm", np.round(warm["errors"], 4), warm["net_used"])
    assert all(warm["net_used"])
    reached = []
    for r in range(len(wls)):
        # ahead over the first three sweeps (the gain fades as both solvers
        # approach the noise floor of the smallest reconstruction)
        assert all(w < p for w, p in zip(warm["errors"][r][:3], plain["errors"][r][:3])), r
        target = plain["errors"][r][2]  # the plain batch after three sweeps
        reached.append(next((k for k, e in enumerate(warm["errors"][r]) if e <= target), len(warm["errors"][r])))
    assert sum(reached) < 2 * len(wls), reached  # fewer sweeps in all than the plain batch's three each
