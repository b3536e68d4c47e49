"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars:
* MLP table: FP64 on both sides, |diff| <= 1e-12 (c2, c4 scaled by 2R).
* Interior MLP nodes (Q20) and voxel index lists: bit-exact against the
  oracle's FP32-order node mode; run counts s_j bit-exact.
* Chords: |l_gpu - l_oracle| <= 1e-5 * max(l, h_min).
* DROP image after the fixed sweeps: |x_gpu - x_oracle| <= 1e-3 * max(|x|, 1).
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


def _cmp_rows(oracle, g, rec, ctx, first, count, hmin):
    rp, vox, ln, nodes = ctx.rows(first, count, with_nodes=True)
    rp, vox, ln, nodes = rp.cpu().numpy(), vox.cpu().numpy(), ln.cpu().numpy(), nodes.cpu().numpy()
    orp, ovox, oln = oracle.rows(g, rec, first, count, mode=oracle.MODE_FP32)
    onodes = oracle.nodes(g, rec, first, count, mode=oracle.MODE_FP32)
    assert np.array_equal(nodes, onodes)
    assert np.array_equal(rp, orp)
    assert np.array_equal(vox, ovox)
    err = np.abs(ln.astype(np.float64) - oln)
    assert np.all(err <= 1e-5 * np.maximum(oln, hmin)), err.max()
    return rp, vox, ln


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_mlp_table_matches_oracle(pct, oracle, gi):
    g = [S.Grid(32, 32, 32, 2.0, 2.0, 2.0), S.Grid(160, 160, 64, 1.25, 1.25, 1.25),
         S.Grid(200, 200, 48, 1.0, 1.0, 2.0)][gi]
    with pct.Context(g, n_blocks=1) as ctx:
        tab = ctx.mlp_table()
    ref = oracle.mlp_table(g)
    scale = np.array([1.0, 2 * g.radius, 1.0, 2 * g.radius])
    assert tab.shape == ref.shape
    assert np.abs((tab - ref) / scale).max() <= 1e-12
    R, du, K, E = oracle.geom_info(g)
    with pct.Context(g, n_blocks=1) as ctx:
        assert (ctx.K, ctx.E) == (K, E) and abs(ctx.du - du) < 1e-15 and abs(ctx.R - R) < 1e-15


@pytest.mark.parametrize("n", [1, 127, 129, 3001])
def test_rows_bit_exact_tiny(pct, oracle, n):
    wl = S.tiny_workload(n, seed=7)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=1) as ctx:
        ctx.load(rec)
        _cmp_rows(oracle, wl.grid, rec, ctx, 0, n, 2.0)


@pytest.mark.parametrize("sort", [True, False])
def test_rows_bit_exact_head(pct, oracle, sort):
    wl = S.head_workload(4000, seed=8)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=4, flags=0 if sort else pct.FLAG_NO_SORT) as ctx:
        ctx.load(rec)
        _cmp_rows(oracle, wl.grid, rec, ctx, 0, 4000, 1.25)
        # a ragged interior range
        _cmp_rows(oracle, wl.grid, rec, ctx, 1237, 333, 1.25)


def test_rows_special_paths(pct, oracle):
    # axis-aligned, face-aligned, edge-diagonal and grid-missing protons
    g = S.Grid(32, 32, 32, 2.0, 2.0, 2.0)
    c45 = np.float32(np.sqrt(0.5))
    recs = []
    for (c, s), t, v in [((1, 0), 3.3, -7.1), ((0, 1), 0.0, 0.0), ((-1, 0), 0.0, 20.0), ((c45, c45), 0.0, 5.5),
                         ((-c45, -c45), 0.0, -5.5), ((1, 0), 10.0, 40.0)]:
        r = S.straight_records(g, [t], [v], [0.0], [0.0], [0.0])
        r["cphi"][:] = np.float32(c)
        r["sphi"][:] = np.float32(s)
        recs.append(r)
    rec = S.concat(recs)
    with pct.Context(g, n_blocks=1) as ctx:
        ctx.load(rec)
        rp, vox, ln = _cmp_rows(oracle, g, rec, ctx, 0, len(recs), 2.0)
    assert rp[-1] - rp[-2] == 0  # v = 40 mm passes above the 64 mm tall grid


def test_block_counts_bit_exact(pct, oracle):
    wl = S.tiny_workload(20_000, seed=9)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=3) as ctx:
        ctx.load(rec)
        for b in range(3):
            got = ctx.block_counts(b).cpu().numpy().astype(np.float64)
            assert np.array_equal(got, oracle.block_counts(wl.grid, rec, 3, b, mode=oracle.MODE_FP32))


def _drop_parity(pct, oracle, wl, n_blocks, n_sweeps, lam=1.0, x0=None, flags=0):
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=n_blocks, lam=lam, flags=flags) as ctx:
        ctx.load(rec)
        if x0 is not None:
            ctx.set_x0(x0)
        ctx.iterate(n_sweeps)
        x = ctx.get_rsp().astype(np.float64)
    xo = oracle.drop(wl.grid, rec, n_blocks, n_sweeps, lam=lam, x0=x0, mode=oracle.MODE_FP32)
    err = np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)
    assert err.max() <= 1e-3, (err.max(), int(err.argmax()))
    return x, xo


@pytest.mark.parametrize("sort", [True, False])
def test_drop_parity_tiny_workload(pct, oracle, sort):
    # 32^3 water cylinder, 100k protons, 10 blocks, 10 sweeps
    _drop_parity(pct, oracle, S.tiny_workload(100_000), 10, 10, flags=0 if sort else pct.FLAG_NO_SORT)


@pytest.mark.parametrize("lam,B,n", [(0.5, 7, 10_007), (1.9, 1, 5_000)])
def test_drop_parity_ragged_blocks(pct, oracle, lam, B, n):
    _drop_parity(pct, oracle, S.tiny_workload(n, seed=31), B, 3, lam=lam)


def test_drop_parity_with_x0(pct, oracle):
    wl = S.tiny_workload(20_000, seed=32)
    x0 = S.voxelize(wl.phantom(), wl.grid).astype(np.float32) * 0.9
    _drop_parity(pct, oracle, wl, 5, 2, x0=x0)


def test_drop_parity_head_subset(pct, oracle):
    wl = S.head_workload(200_000, seed=33)
    _drop_parity(pct, oracle, wl, 10, 2)


def test_invalid_records_are_rejected(pct):
    wl = S.tiny_workload(1000, seed=10)
    rec = S.make_histories(wl)
    bad = {k: v.copy() for k, v in rec.items()}
    bad["st0"][17] = 0.7
    bad["wepl"][400] = np.nan
    with pct.Context(wl.grid, n_blocks=2) as ctx:
        with pytest.raises(pct.PctError) as ei:
            ctx.load(bad)
        assert ei.value.code == -2 and ctx.first_bad == 17
        with pytest.raises(pct.PctError) as ei:
            ctx.iterate(1)
        assert ei.value.code == -7
        ctx.load(rec)  # a valid load afterwards works
        ctx.iterate(1)
        ctx.sync()
    with pct.Context(wl.grid, n_blocks=2000) as ctx:
        with pytest.raises(pct.PctError):
            ctx.load(rec)  # fewer histories than blocks


def test_device_borrow_equals_host_copy(pct):
    import torch

    wl = S.tiny_workload(5000, seed=11)
    rec = S.make_histories(wl)
    trec = {k: torch.from_numpy(v).cuda() for k, v in rec.items()}
    out = []
    for r, borrow in ((rec, False), (trec, True), (trec, False)):
        with pct.Context(wl.grid, n_blocks=5, flags=pct.FLAG_NO_SORT) as ctx:
            ctx.load(r, borrow=borrow)
            ctx.iterate(2)
            out.append(ctx.get_rsp())
    # same inputs, same launch order: only atomic ordering differs
    assert np.abs(out[0] - out[1]).max() <= 1e-4 * max(1.0, np.abs(out[0]).max())
    assert np.abs(out[0] - out[2]).max() <= 1e-4 * max(1.0, np.abs(out[0]).max())


@pytest.mark.parametrize("kahan", [True, False])
def test_projection_and_residual_match_oracle(pct, oracle, kahan):
    # a_i.x (Sec. 2: the model WEPL) with the fused kernel's arithmetic against
    # the oracle's FP64 sum over the same rows (FP32-order nodes)
    wl = S.head_workload(20_000, seed=61)
    g = wl.grid
    rec = S.make_histories(wl)
    x0 = S.voxelize(wl.phantom(), g, ss=2).astype(np.float32)
    flags = 0 if kahan else pct.FLAG_NO_KAHAN
    with pct.Context(g, n_blocks=4, flags=flags) as ctx:
        ctx.load(rec)
        ctx.set_x0(x0)
        y = ctx.project(0, 20_000).cpu().numpy().astype(np.float64)
        y2 = ctx.project(777, 1000).cpu().numpy().astype(np.float64)
        rr = ctx.residual()
        rr7 = ctx.residual(7)
    yo = oracle.project(g, rec, x0.astype(np.float64), mode=oracle.MODE_FP32)
    tol = 1e-5 if kahan else 1e-4
    assert np.all(np.abs(y - yo) <= tol * np.maximum(np.abs(yo), 1.0))
    assert np.array_equal(y2, y[777:1777])
    ro = float(((rec["wepl"].astype(np.float64) - yo) ** 2).sum())
    assert abs(rr - ro) <= 1e-4 * ro
    # a 1/7 sample estimates the same sum (stored order is grouped by angle)
    assert abs(7 * rr7 - ro) <= 0.1 * ro


@pytest.mark.parametrize("strings,blocks,sweeps", [(10, 10, 5), (3, 3, 2), (4, 12, 3), (3, 7, 2)])
def test_carp_parity(pct, oracle, strings, blocks, sweeps):
    # CARP (Sec. 2.2): strings of DROP blocks swept from a common x, then
    # component averaging
    wl = S.tiny_workload(60_000, seed=71)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=blocks, flags=pct.FLAG_CARP, carp_strings=strings) as ctx:
        ctx.load(rec)
        ctx.iterate(sweeps)
        x = ctx.get_rsp().astype(np.float64)
    xo = oracle.carp(wl.grid, rec, strings, sweeps, mode=oracle.MODE_FP32, n_blocks=blocks)
    err = np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)
    assert err.max() <= 1e-3, err.max()


@pytest.mark.parametrize("carp", [False, True])
def test_tvs_parity(pct, oracle, carp):
    # total-variation superiorization (Sec. 4.2) before every DROP block or
    # every CARP iteration, against the oracle's reading
    wl = S.tiny_workload(30_000, seed=95)
    rec = S.make_histories(wl)
    flags = pct.FLAG_CARP if carp else 0
    with pct.Context(wl.grid, n_blocks=4, flags=flags, tvs_beta0=0.05, tvs_alpha=0.99, tvs_eps=1e-4,
                     tvs_tries=4, carp_strings=2) as ctx:
        ctx.load(rec)
        ctx.iterate(3)
        x = ctx.get_rsp().astype(np.float64)
    xo = oracle.solve_tvs(wl.grid, rec, 4, 3, carp=2 if carp else 0, beta0=0.05, alpha=0.99, eps=1e-4, tries=4,
                          mode=oracle.MODE_FP32)
    err = np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)
    assert err.max() <= 1e-3, err.max()
    plain = oracle.carp(wl.grid, rec, 2, 3, n_blocks=4) if carp else oracle.drop(wl.grid, rec, 4, 3)
    assert oracle.tv_value(wl.grid, x) < oracle.tv_value(wl.grid, plain)


def test_host_load_through_two_staging_slots_matches_a_device_copy(pct, oracle):
    # Host records pass through two staging slots (block b + 1 copied while
    # block b is validated and ordered). Seven ragged blocks reuse each slot
    # three times: the rows in load order and the run counts equal those of a
    # device-copy load and the oracle's, and a bad record in the last block is
    # found.
    import torch

    wl = S.tiny_workload(7003, seed=16)
    g = wl.grid
    rec = S.make_histories(wl)
    hmin = min(g.hx, g.hy, g.hz)
    with pct.Context(g, n_blocks=7) as host, pct.Context(g, n_blocks=7) as dev:
        host.load(rec)
        dev.load({k: torch.from_numpy(v).cuda() for k, v in rec.items()})
        a = _cmp_rows(oracle, g, rec, host, 0, wl.n, hmin)
        b = [t.cpu().numpy() for t in dev.rows(0, wl.n)]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
        host.iterate(2)
        dev.iterate(2)
        x, y = host.get_rsp(), dev.get_rsp()
        assert np.abs(x - y).max() <= 1e-4 * max(1.0, np.abs(y).max())
        bad = {k: v.copy() for k, v in rec.items()}
        bad["sv2"][wl.n - 2] = np.inf
        with pytest.raises(pct.PctError) as ei:
            host.load(bad)
        assert ei.value.code == -2 and host.first_bad == wl.n - 2
        host.load(rec)
        host.iterate(2)
        z = host.get_rsp()
    xo = oracle.drop(g, rec, 7, 2, mode=oracle.MODE_FP32)
    assert np.max(np.abs(z - xo) / np.maximum(np.abs(xo), 1.0)) <= 1e-3


def test_empty_load_is_rejected(pct):
    wl = S.tiny_workload(10, seed=12)
    rec = {k: v[:0] for k, v in S.make_histories(wl).items()}
    with pct.Context(wl.grid, n_blocks=1) as ctx:
        with pytest.raises(pct.PctError) as ei:
            ctx.load(rec)
        assert ei.value.code == -1


def test_reloads_of_other_sizes_match_fresh_contexts(pct, oracle):
    # One context reloaded with growing and shrinking sets (its buffers are
    # kept and grown across loads; the first sweep after each load counts the
    # block weights) gives the result of a fresh context each time.
    wl = S.tiny_workload(20_000, seed=13)
    g = wl.grid
    full = S.make_histories(wl)
    with pct.Context(g, n_blocks=4) as reused:
        for n in (5000, 20_000, 3001, 12_000):
            rec = S.subset(full, slice(0, n))
            reused.load(rec)
            reused.iterate(2)
            a = reused.get_rsp()
            with pct.Context(g, n_blocks=4) as fresh:
                fresh.load(rec)
                fresh.iterate(2)
                b = fresh.get_rsp()
            assert np.abs(a - b).max() <= 1e-4 * max(1.0, np.abs(b).max()), n
            # and both follow the oracle
            xo = oracle.drop(g, rec, 4, 2, mode=oracle.MODE_FP32)
            assert np.max(np.abs(a - xo) / np.maximum(np.abs(xo), 1.0)) <= 1e-3, n


def test_borrowed_reload_with_moved_arrays_matches_fresh_context(pct):
    # A borrowed, unsorted reload of the same size that keeps the t0 array but
    # moves the ten others: the sweep graphs captured every record pointer, so
    # the reused context must rebuild them and match a fresh context. The
    # first set stays alive throughout.
    import torch

    wl = S.tiny_workload(6000, seed=14)
    a = {k: torch.from_numpy(v).cuda() for k, v in S.make_histories(wl).items()}
    other = S.make_histories(S.tiny_workload(6000, seed=15))
    b = {k: (a[k] if k == "t0" else torch.from_numpy(v).cuda()) for k, v in other.items()}
    with pct.Context(wl.grid, n_blocks=3, flags=pct.FLAG_NO_SORT) as reused:
        reused.load(a, borrow=True)
        reused.iterate(2)
        reused.load(b, borrow=True)
        reused.iterate(2)
        x = reused.get_rsp()
    with pct.Context(wl.grid, n_blocks=3, flags=pct.FLAG_NO_SORT) as fresh:
        fresh.load(b, borrow=True)
        fresh.iterate(2)
        y = fresh.get_rsp()
    assert np.abs(x - y).max() <= 1e-4 * max(1.0, np.abs(y).max())


def test_sweeps_on_a_side_stream_are_ordered_before_later_calls(pct):
    # sweeps queued on another torch stream, then the image read on the default
    # stream: switching streams waits for the old one, so the read sees all sweeps
    import torch

    wl = S.tiny_workload(20_000, seed=16)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=4) as ref:
        ref.load(rec)
        ref.iterate(3)
        a = ref.get_rsp()
    side = torch.cuda.Stream()
    with pct.Context(wl.grid, n_blocks=4) as ctx:
        ctx.load(rec)
        with torch.cuda.stream(side):
            ctx.iterate(3)
        b = ctx.get_rsp()
    assert np.abs(a - b).max() <= 1e-4 * max(1.0, np.abs(a).max())


def test_block_weights_formed_ahead_give_the_same_image(pct, oracle):
    # pct_block_weights forms every block's s_j before the first sweep (the
    # sweep then runs without counting); the image is the oracle's either way
    wl = S.tiny_workload(30_000, seed=34)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=4) as ctx:
        with pytest.raises(pct.PctError):
            ctx.block_weights()  # nothing loaded yet
        ctx.load(rec)
        ctx.block_weights()
        ctx.block_weights()  # formed already: no-op
        for b in range(4):
            got = ctx.block_counts(b).cpu().numpy().astype(np.float64)
            assert np.array_equal(got, oracle.block_counts(wl.grid, rec, 4, b, mode=oracle.MODE_FP32))
        ctx.iterate(3)
        x = ctx.get_rsp().astype(np.float64)
    xo = oracle.drop(wl.grid, rec, 4, 3, mode=oracle.MODE_FP32)
    err = np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)
    assert err.max() <= 1e-3, err.max()
