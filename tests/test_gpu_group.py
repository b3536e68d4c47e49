"""GPU parity of the group walk (2, 4, 8, 16 or 32 lanes per history, the
threads_per_proton setting) against the FP64 oracle, through the C ABI.

The group walk splits a history's MLP segments over the lanes and merges the
runs across them; its rows must be those of the oracle exactly as for the
one-lane walk: Q20 nodes, row_ptr and voxel index lists bit-exact against the
oracle's FP32-order nodes, chords within 1e-5 * max(l, h_min), DROP images
within 1e-3 * max(|x|, 1) after the fixed sweeps (the first sweep's fused
kernel also forms the block weights s_j, which the image depends on)."""
import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S
from paper_1707_05014_gb300 import warmstart as W

pytestmark = pytest.mark.gpu

RSP_TOL = 1e-3
CHORD_TOL = 1e-5
LANES = [2, 4, 8, 16, 32]


@pytest.fixture(scope="module")
def pct():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1707_05014_gb300 import build, pct as P

    build.build()
    return P


def _cmp_rows(oracle, g, rec, ctx, first, count, node_step=0.0):
    hmin = min(g.hx, g.hy, g.hz)
    rp, vox, ln, nodes = (t.cpu().numpy() for t in ctx.rows(first, count, with_nodes=True))
    sub = S.subset(rec, slice(first, first + count))
    assert np.array_equal(nodes, oracle.nodes(g, sub, mode=oracle.MODE_FP32, node_step=node_step))
    orp, ovox, oln = oracle.rows(g, sub, mode=oracle.MODE_FP32, node_step=node_step)
    assert np.array_equal(rp, orp), int(np.argmax(rp != orp))
    assert np.array_equal(vox, ovox), int(np.argmax(vox != ovox))
    err = np.abs(ln.astype(np.float64) - oln)
    assert np.all(err <= CHORD_TOL * np.maximum(oln, hmin)), err.max()
    return rp


@pytest.mark.parametrize("lanes", LANES)
@pytest.mark.parametrize("n", [1, 31, 129, 3001])
def test_group_rows_bit_exact_tiny(pct, oracle, lanes, n):
    wl = S.tiny_workload(n, seed=7)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=1, lanes=lanes) as ctx:
        ctx.load(rec)
        _cmp_rows(oracle, wl.grid, rec, ctx, 0, n)


@pytest.mark.parametrize("lanes", LANES)
def test_group_rows_bit_exact_head(pct, oracle, lanes):
    wl = S.head_workload(4000, seed=8)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=4, lanes=lanes) as ctx:
        ctx.load(rec)
        _cmp_rows(oracle, wl.grid, rec, ctx, 0, 4000)
        _cmp_rows(oracle, wl.grid, rec, ctx, 1237, 333)  # a ragged interior range


@pytest.mark.parametrize("lanes", LANES)
def test_group_rows_bit_exact_on_the_anisotropic_grid(pct, oracle, lanes):
    g = W.training_grid()  # 200 x 200 x 48 of 1 x 1 x 2 mm
    wl = W.head_workload(g, 4000, seed=83)
    rec = S.make_histories(wl)
    with pct.Context(g, n_blocks=4, lanes=lanes) as ctx:
        ctx.load(rec)
        _cmp_rows(oracle, g, rec, ctx, 0, 4000)


@pytest.mark.parametrize("lanes", [8, 32])
def test_group_rows_special_paths(pct, oracle, lanes):
    # axis-aligned, face-aligned, edge-diagonal and grid-missing protons: exact
    # ties between crossings of two and three axes, nodes on faces
    g = S.Grid(32, 32, 32, 2.0, 2.0, 2.0)
    c45 = np.float32(np.sqrt(0.5))
    recs = []
    for (c, s), t, v in [((1, 0), 3.3, -7.1), ((0, 1), 0.0, 0.0), ((-1, 0), 0.0, 20.0), ((c45, c45), 0.0, 5.5),
                         ((-c45, -c45), 0.0, -5.5), ((1, 0), 10.0, 40.0), ((c45, c45), 0.0, 0.0),
                         ((0, -1), 2.0, 4.0)]:
        r = S.straight_records(g, [t], [v], [0.0], [0.0], [0.0])
        r["cphi"][:] = np.float32(c)
        r["sphi"][:] = np.float32(s)
        recs.append(r)
    rec = S.concat(recs)
    with pct.Context(g, n_blocks=1, lanes=lanes) as ctx:
        ctx.load(rec)
        rp = _cmp_rows(oracle, g, rec, ctx, 0, len(recs))
    assert rp[6] - rp[5] == 0  # v = 40 mm passes above the 64 mm tall grid


@pytest.mark.parametrize("lanes", [16])
@pytest.mark.parametrize("step", [1.25, 3.0])
def test_group_rows_at_long_node_steps(pct, oracle, lanes, step):
    # segments longer than a voxel: the group hands the history to one lane
    wl = S.head_workload(1000, seed=81)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=2, node_step=step, lanes=lanes) as ctx:
        ctx.load(rec)
        _cmp_rows(oracle, wl.grid, rec, ctx, 0, 1000, node_step=step)


def _drop(pct, oracle, g, rec, n_blocks, n_sweeps, lanes, flags=0, node_step=0.0):
    with pct.Context(g, n_blocks=n_blocks, flags=flags, node_step=node_step, lanes=lanes) as ctx:
        ctx.load(rec)
        ctx.iterate(n_sweeps)
        x = ctx.get_rsp().astype(np.float64)
    xo = oracle.drop(g, rec, n_blocks, n_sweeps, mode=oracle.MODE_FP32, node_step=node_step)
    err = np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)
    assert err.max() <= RSP_TOL, (err.max(), int(err.argmax()))
    return x


@pytest.mark.parametrize("lanes", LANES)
def test_group_drop_parity_tiny(pct, oracle, lanes):
    wl = S.tiny_workload(100_000)
    _drop(pct, oracle, wl.grid, S.make_histories(wl), 10, 10, lanes)


@pytest.mark.parametrize("lanes", [8, 32])
def test_group_drop_parity_head_subset_plain_sum(pct, oracle, lanes):
    wl = S.head_workload(200_000, seed=33)
    _drop(pct, oracle, wl.grid, S.make_histories(wl), 10, 2, lanes, flags=pct.FLAG_NO_KAHAN)


@pytest.mark.parametrize("lanes", LANES)
def test_group_drop_parity_on_the_anisotropic_grid(pct, oracle, lanes):
    g = W.training_grid()
    wl = W.head_workload(g, 200_000, seed=84, n_blocks=50)
    _drop(pct, oracle, g, S.make_histories(wl), 50, 2, lanes)


def test_group_drop_parity_at_a_long_node_step(pct, oracle):
    wl = S.head_workload(50_000, seed=82)
    _drop(pct, oracle, wl.grid, S.make_histories(wl), 5, 2, 32, node_step=3.0)


def test_group_with_hull_runs_the_one_lane_kernels(pct):
    # a hull is not walked by the group: the context falls back to one lane per
    # history and gives the one-lane image (up to the order of the float
    # atomics, which no run fixes)
    wl = S.head_workload(20_000, seed=85)
    rec = S.make_histories(wl)
    xs = []
    for lanes in (1, 32):
        with pct.Context(wl.grid, n_blocks=2, lanes=lanes) as ctx:
            ctx.load(rec)
            ctx.carve_hull(1.0, 1)
            ctx.iterate(1)
            xs.append(ctx.get_rsp())
    err = np.abs(xs[0].astype(np.float64) - xs[1]) / np.maximum(np.abs(xs[0]), 1.0)
    assert err.max() <= 1e-5, err.max()


def test_lane_counts_outside_the_supported_set_are_rejected(pct):
    g = S.Grid(8, 8, 8, 2.0, 2.0, 2.0)
    for lanes in (3, 7, 64):
        with pytest.raises(pct.PctError):
            pct.Context(g, n_blocks=1, lanes=lanes)
