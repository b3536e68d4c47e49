"""GPU parity at the library's size limits and in degenerate cases, through the
C ABI against the FP64 oracle (FP32-order nodes): the largest MLP node count
(K + 1 = 2048, the shared-memory table's limit), the largest grid axis (512
voxels, here along z: 2.1M voxels), and histories that all miss the grid
(empty rows: no update, no NaN).
Bars as in the other parity tests: Q20 nodes, row_ptr and index lists
bit-exact, chords within 1e-5 * max(l, h_min), images within 1e-3 * max(|x|, 1)."""
import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

RSP_TOL = 1e-3
CHORD_TOL = 1e-5


@pytest.fixture(scope="module")
def pct():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1707_05014_gb300 import build, pct as P

    build.build()
    return P


def _cmp_rows(oracle, g, rec, ctx, node_step):
    n = len(rec["t0"])
    hmin = min(g.hx, g.hy, g.hz)
    rp, vox, ln, nodes = (t.cpu().numpy() for t in ctx.rows(0, n, with_nodes=True))
    assert np.array_equal(nodes, oracle.nodes(g, rec, mode=oracle.MODE_FP32, node_step=node_step))
    orp, ovox, oln = oracle.rows(g, rec, mode=oracle.MODE_FP32, node_step=node_step)
    assert np.array_equal(rp, orp)
    assert np.array_equal(vox, ovox)
    err = np.abs(ln.astype(np.float64) - oln)
    assert np.all(err <= CHORD_TOL * np.maximum(oln, hmin)), err.max()
    return rp


@pytest.mark.parametrize("lanes", [1, 32])
def test_rows_and_drop_at_the_largest_node_count(pct, oracle, lanes):
    wl = S.tiny_workload(2000, seed=61)
    g = wl.grid
    step = 2.0 * g.radius / 2047.0  # K = 2047: K + 1 = 2048 nodes
    rec = S.make_histories(wl)
    with pct.Context(g, n_blocks=2, node_step=step, lanes=lanes) as ctx:
        assert ctx.K == 2047
        ctx.load(rec)
        _cmp_rows(oracle, g, rec, ctx, step)
        ctx.iterate(2)
        x = ctx.get_rsp().astype(np.float64)
    xo = oracle.drop(g, rec, 2, 2, mode=oracle.MODE_FP32, node_step=step)
    err = np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)
    assert err.max() <= RSP_TOL, err.max()


def test_one_node_more_than_the_table_holds_is_rejected(pct):
    g = S.Grid(32, 32, 32, 2.0, 2.0, 2.0)
    with pytest.raises(pct.PctError):
        pct.Context(g, n_blocks=1, node_step=2.0 * g.radius / 2048.0)  # K + 1 = 2049


@pytest.mark.parametrize("lanes", [1, 16])
def test_rows_and_drop_on_the_largest_grid_axis(pct, oracle, lanes):
    # 64 x 64 x 512 voxels of 1 mm (2.1M voxels; voxel indices up to 2^21), a
    # water cylinder of r = 25 mm along z, entry heights over +-250 mm
    g = S.Grid(64, 64, 512, 1.0, 1.0, 1.0)
    wl = S.Workload("axis512", g, 3000, 62, 0, 30.0, 250.0, 3, 2, "water")
    rec = S.make_histories(wl)
    with pct.Context(g, n_blocks=3, lanes=lanes) as ctx:
        ctx.load(rec)
        rp = _cmp_rows(oracle, g, rec, ctx, 0.0)
        assert rp[-1] > 0
        ctx.iterate(2)
        x = ctx.get_rsp().astype(np.float64)
    xo = oracle.drop(g, rec, 3, 2, mode=oracle.MODE_FP32)
    err = np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)
    assert err.max() <= RSP_TOL, err.max()
    with pytest.raises(pct.PctError):
        pct.Context(S.Grid(64, 64, 513, 1.0, 1.0, 1.0), n_blocks=1)


@pytest.mark.parametrize("lanes", [1, 8])
def test_histories_that_all_miss_the_grid(pct, oracle, lanes):
    # every path passes above the grid: empty rows, no update, finite image
    g = S.Grid(32, 32, 32, 2.0, 2.0, 2.0)
    rng = np.random.Generator(np.random.Philox(63))
    n = 500
    rec = S.straight_records(g, rng.uniform(-25, 25, n), rng.uniform(40, 60, n), rng.normal(0, 1e-3, n),
                             np.zeros(n), rng.uniform(0, 2 * np.pi, n))
    with pct.Context(g, n_blocks=2, lanes=lanes) as ctx:
        ctx.load(rec)
        rp = _cmp_rows(oracle, g, rec, ctx, 0.0)
        assert rp[-1] == 0
        ctx.iterate(2)
        x = ctx.get_rsp()
    assert np.all(x == 0.0)
