"""Parity at the bench's full size: the 50M-history head workload (160 x 160 x 64
grid of 1.25 mm, 10 blocks), loaded as bench.py loads it (device-generated
records, blocks ordered on the GPU). The oracle checks sampled histories one
by one across the whole index range -- MLP nodes, voxel index lists (bit-exact)
and chords -- and a_i.x after a full sweep; a property that holds at any size
(the data residual falls over a sweep) covers the rest."""
import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1707_05014_gb300 import build, pct

    build.build()
    wl = S.head_workload(50_000_000, seed=2)
    rec = S.make_histories_device(wl)
    ctx = pct.Context(wl.grid, n_blocks=wl.n_blocks)
    ctx.load(rec, borrow=True)
    starts = [0, 4_999_937, 12_345_678, 25_000_000, 37_777_777, 49_999_800]
    host = S.concat([{k: v[s:s + 200].cpu().numpy() for k, v in rec.items()} for s in starts])
    yield wl, ctx, starts, host
    ctx.close()


def test_sampled_rows_bit_exact_at_full_size(full, oracle):
    wl, ctx, starts, host = full
    g = wl.grid
    for q, s in enumerate(starts):
        rp, vox, ln, nodes = (t.cpu().numpy() for t in ctx.rows(s, 200, with_nodes=True))
        sub = S.subset(host, slice(200 * q, 200 * q + 200))
        orp, ovox, oln = oracle.rows(g, sub, mode=oracle.MODE_FP32)
        assert np.array_equal(nodes, oracle.nodes(g, sub, mode=oracle.MODE_FP32))
        assert np.array_equal(rp, orp) and np.array_equal(vox, ovox)
        assert np.all(np.abs(ln - oln) <= 1e-5 * np.maximum(oln, g.hx))


def test_full_sweep_projection_and_residual(full, oracle):
    wl, ctx, starts, host = full
    g = wl.grid
    r0 = ctx.residual(64)
    ctx.iterate(1)
    r1 = ctx.residual(64)
    assert r1 < 0.5 * r0  # one sweep from x = 0 fits most of the data
    x = ctx.get_rsp().astype(np.float64)
    assert np.isfinite(x).all()
    for q, s in enumerate(starts):
        y = ctx.project(s, 200).cpu().numpy().astype(np.float64)
        yo = oracle.project(g, S.subset(host, slice(200 * q, 200 * q + 200)), x, mode=oracle.MODE_FP32)
        assert np.all(np.abs(y - yo) <= 1e-5 * np.maximum(np.abs(yo), 1.0))


def test_sampled_hull_rows_bit_exact_at_full_size(full, oracle):
    # the same loaded 50M histories with the voxelised head as object hull:
    # hull ranges, nodes and index lists of the samples match the oracle's
    # hull path, and a sweep with the hull still fits the data
    wl, ctx, starts, host = full
    g = wl.grid
    hull = (S.voxelize(wl.phantom(), g, ss=1) > 0.5).astype(np.uint8)
    ctx.set_hull(hull)
    try:
        for q, s in enumerate(starts[::2]):
            sub = S.subset(host, slice(400 * q, 400 * q + 200))
            rng = ctx.hull_ranges(s, 200)
            assert np.array_equal(rng, oracle.hull_ranges(g, sub, hull, mode=oracle.MODE_FP32))
            rp, vox, ln, nodes = (t.cpu().numpy() for t in ctx.rows(s, 200, with_nodes=True))
            assert np.array_equal(nodes, oracle.nodes(g, sub, mode=oracle.MODE_FP32, hull=hull))
            orp, ovox, oln = oracle.rows(g, sub, mode=oracle.MODE_FP32, hull=hull)
            assert np.array_equal(rp, orp) and np.array_equal(vox, ovox)
            assert np.all(np.abs(ln - oln) <= 1e-5 * np.maximum(oln, g.hx))
        ctx.set_x0(np.zeros(g.m, np.float32))
        r0 = ctx.residual(64)
        ctx.iterate(1)
        assert ctx.residual(64) < 0.5 * r0
    finally:
        ctx.set_hull(None)
