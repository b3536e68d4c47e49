"""Parity at the largest workload's full size: 1e9 histories on the 200 x 200 x 48
grid of 1 x 1 x 2 mm voxels (1.92M voxels), 50 blocks, loaded as bench.py
loads it (device-generated records, 44 GB, blocks ordered on the GPU). The
oracle checks sampled histories one by one across the whole index range (MLP
nodes and voxel index lists bit-exact, chords within 1e-5) and a_i.x after a
full sweep; the data residual falling over the sweep covers the rest."""
import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

STARTS = [0, 19_999_950, 123_456_789, 500_000_000, 777_777_777, 999_999_800]


@pytest.fixture(scope="module")
def full():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1707_05014_gb300 import build, pct

    build.build()
    wl = S.head200_workload()
    rec = S.make_histories_device(wl)
    host = S.concat([{k: v[s:s + 200].cpu().numpy() for k, v in rec.items()} for s in STARTS])
    ctx = pct.Context(wl.grid, n_blocks=wl.n_blocks)
    ctx.load(rec)  # a device copy, ordered within each block
    del rec
    torch.cuda.empty_cache()
    yield wl, ctx, host
    ctx.close()
    torch.cuda.empty_cache()


def test_sampled_rows_bit_exact_at_1e9(full, oracle):
    wl, ctx, host = full
    g = wl.grid
    for q, s in enumerate(STARTS):
        rp, vox, ln, nodes = (t.cpu().numpy() for t in ctx.rows(s, 200, with_nodes=True))
        sub = S.subset(host, slice(200 * q, 200 * q + 200))
        orp, ovox, oln = oracle.rows(g, sub, mode=oracle.MODE_FP32)
        assert np.array_equal(nodes, oracle.nodes(g, sub, mode=oracle.MODE_FP32))
        assert np.array_equal(rp, orp) and np.array_equal(vox, ovox)
        assert np.all(np.abs(ln - oln) <= 1e-5 * np.maximum(oln, min(g.hx, g.hy, g.hz)))


def test_full_sweep_at_1e9_projection_and_residual(full, oracle):
    wl, ctx, host = full
    g = wl.grid
    r0 = ctx.residual(256)
    ctx.iterate(1)
    r1 = ctx.residual(256)
    assert r1 < 0.5 * r0
    x = ctx.get_rsp().astype(np.float64)
    assert np.isfinite(x).all()
    for q, s in enumerate(STARTS):
        y = ctx.project(s, 200).cpu().numpy().astype(np.float64)
        yo = oracle.project(g, S.subset(host, slice(200 * q, 200 * q + 200)), x, mode=oracle.MODE_FP32)
        assert np.all(np.abs(y - yo) <= 1e-5 * np.maximum(np.abs(yo), 1.0))
