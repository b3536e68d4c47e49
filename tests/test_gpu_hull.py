"""GPU parity of the object-hull path (pct_set_hull / pct_carve_hull) through
the C ABI against the FP64 oracle's hull path.

Bars as for the plane-to-plane path: layer tables FP64 within 1e-12 (c2, c4
scaled by the layer thickness); hull ranges, interior Q20 nodes, voxel index
lists, run counts and the carved mask bit-exact against the oracle's FP32
node order; chords within 1e-5 * max(l, h_min); DROP/CARP images within
1e-3 * max(|x|, 1) after the fixed sweeps.
"""
import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pct():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1707_05014_gb300 import build, pct as P

    build.build()
    return P


def _mask(wl):
    return (S.voxelize(wl.phantom(), wl.grid, ss=1) > 0.5).astype(np.uint8)


@pytest.mark.parametrize("frac", [0.01, 0.37, 0.8, 1.0])
def test_layer_tables_match_oracle(pct, oracle, frac):
    g = S.Grid(160, 160, 64, 1.25, 1.25, 1.25)
    with pct.Context(g, n_blocks=1) as ctx:
        n = max(1, int(frac * ctx.K))
        got = ctx.mlp_table_n(n)
        plane = ctx.mlp_table()
    ref = oracle.mlp_table_n(g, n)
    L = n * oracle.geom_info(g)[1]
    assert np.abs((got - ref) / np.array([1.0, L, 1.0, L])).max() <= 1e-12
    if frac == 1.0:
        assert np.array_equal(got, plane)


def _cmp_hull_rows(pct, oracle, wl, rec, hull, n_blocks, flags, first, count, hmin):
    g = wl.grid
    with pct.Context(g, n_blocks=n_blocks, flags=flags) as ctx:
        ctx.set_hull(hull)
        ctx.load(rec)
        rng = ctx.hull_ranges(first, count)
        rp, vox, ln, nodes = (t.cpu().numpy() for t in ctx.rows(first, count, with_nodes=True))
    orng = oracle.hull_ranges(g, rec, hull, first, count, mode=oracle.MODE_FP32)
    assert np.array_equal(rng, orng)
    onodes = oracle.nodes(g, rec, first, count, mode=oracle.MODE_FP32, hull=hull)
    assert np.array_equal(nodes, onodes)
    orp, ovox, oln = oracle.rows(g, rec, first, count, mode=oracle.MODE_FP32, hull=hull)
    assert np.array_equal(rp, orp) and np.array_equal(vox, ovox)
    err = np.abs(ln.astype(np.float64) - oln)
    assert np.all(err <= 1e-5 * np.maximum(oln, hmin)), err.max()
    return orng


def test_hull_rows_bit_exact_tiny(pct, oracle):
    wl = S.tiny_workload(3001, seed=41)
    rec = S.make_histories(wl)
    rng = _cmp_hull_rows(pct, oracle, wl, rec, _mask(wl), 1, 0, 0, 3001, 2.0)
    _, _, K, _ = oracle.geom_info(wl.grid)
    assert ((rng[:, 0] > 0) & (rng[:, 1] < K)).mean() > 0.5  # most protons use a layer table


@pytest.mark.parametrize("sort", [True, False])
def test_hull_rows_bit_exact_head(pct, oracle, sort):
    wl = S.head_workload(3000, seed=42)
    rec = S.make_histories(wl)
    hull = _mask(wl)
    flags = 0 if sort else pct.FLAG_NO_SORT
    _cmp_hull_rows(pct, oracle, wl, rec, hull, 4, flags, 0, 3000, 1.25)
    _cmp_hull_rows(pct, oracle, wl, rec, hull, 4, flags, 1111, 457, 1.25)


def test_hull_set_after_load_and_removed(pct, oracle):
    wl = S.tiny_workload(5000, seed=43)
    rec = S.make_histories(wl)
    g = wl.grid
    hull = _mask(wl)
    with pct.Context(g, n_blocks=3) as ctx:
        ctx.load(rec)
        ctx.set_hull(hull)
        for b in range(3):
            got = ctx.block_counts(b).cpu().numpy().astype(np.float64)
            assert np.array_equal(got, oracle.block_counts(g, rec, 3, b, mode=oracle.MODE_FP32, hull=hull))
        ctx.set_hull(None)
        got = ctx.block_counts(1).cpu().numpy().astype(np.float64)
        assert np.array_equal(got, oracle.block_counts(g, rec, 3, 1, mode=oracle.MODE_FP32))


def test_carved_hull_bit_exact(pct, oracle):
    wl = S.tiny_workload(20_000, seed=44)
    rec = S.make_histories(wl, noise=0.0)
    g = wl.grid
    with pct.Context(g, n_blocks=2) as ctx:
        ctx.load(rec)
        ctx.carve_hull(wepl_max=1.0, dilate=1)
        got = ctx.get_hull()
        rng = ctx.hull_ranges(0, 500)
    ref = oracle.carve_hull(g, rec, wepl_max=1.0, dilate=1, mode=oracle.MODE_FP32)
    assert np.array_equal(got, ref)
    assert np.array_equal(rng, oracle.hull_ranges(g, rec, ref, 0, 500, mode=oracle.MODE_FP32))


def _hull_solve_parity(pct, oracle, wl, n_blocks, n_sweeps, carp=0):
    rec = S.make_histories(wl)
    hull = _mask(wl)
    kw = dict(flags=pct.FLAG_CARP, carp_strings=carp) if carp else {}
    with pct.Context(wl.grid, n_blocks=n_blocks, **kw) as ctx:
        ctx.set_hull(hull)
        ctx.load(rec)
        ctx.iterate(n_sweeps)
        x = ctx.get_rsp().astype(np.float64)
    if carp:
        xo = oracle.carp(wl.grid, rec, carp, n_sweeps, n_blocks=n_blocks, mode=oracle.MODE_FP32, hull=hull)
    else:
        xo = oracle.drop(wl.grid, rec, n_blocks, n_sweeps, mode=oracle.MODE_FP32, hull=hull)
    err = np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)
    assert err.max() <= 1e-3, (err.max(), int(err.argmax()))


def test_hull_drop_parity_tiny(pct, oracle):
    _hull_solve_parity(pct, oracle, S.tiny_workload(100_000, seed=45), 10, 5)


def test_hull_carp_parity_tiny(pct, oracle):
    _hull_solve_parity(pct, oracle, S.tiny_workload(30_000, seed=46), 8, 2, carp=4)


def test_hull_drop_parity_head_subset(pct, oracle):
    _hull_solve_parity(pct, oracle, S.head_workload(100_000, seed=47), 10, 2)


def test_hull_contexts_are_not_batched(pct):
    wl = S.tiny_workload(2000, seed=48)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=2) as a:
        a.load(rec)
        a.set_hull(_mask(wl))
        with pytest.raises(pct.PctError):
            pct.Batch([a])


def test_hull_set_after_sweeps_is_recounted_by_the_next_sweep(pct, oracle):
    # sweeps without a hull, then a hull: the next sweep recounts the block
    # weights for the hull rows and the image follows the oracle's hull DROP
    wl = S.tiny_workload(20_000, seed=49)
    rec = S.make_histories(wl)
    g = wl.grid
    hull = _mask(wl)
    with pct.Context(g, n_blocks=5) as ctx:
        ctx.load(rec)
        ctx.iterate(2)
        ctx.set_hull(hull)
        ctx.set_x0(np.zeros(g.m, np.float32))
        ctx.iterate(2)
        x = ctx.get_rsp().astype(np.float64)
    xo = oracle.drop(g, rec, 5, 2, mode=oracle.MODE_FP32, hull=hull)
    assert np.max(np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)) <= 1e-3
