"""GPU parity on the configurations the default tests leave out: MLP node
spacings longer than half a voxel (a segment then spans more than one voxel on
an axis, so the walk's multi-face branch runs) and the anisotropic
200 x 200 x 48 grid of 1 x 1 x 2 mm voxels of the 1e9-history workload.

Bars as in the parity tests: Q20 nodes, row_ptr and voxel index lists
bit-exact against the oracle's FP32-order nodes; chords within
1e-5 * max(l, h_min); DROP images within 1e-3 * max(|x|, 1)."""
import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S
from paper_1707_05014_gb300 import warmstart as W

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


def _cmp_rows(oracle, g, rec, ctx, first, count, node_step=0.0):
    hmin = min(g.hx, g.hy, g.hz)
    rp, vox, ln, nodes = (t.cpu().numpy() for t in ctx.rows(first, count, with_nodes=True))
    sub = S.subset(rec, slice(first, first + count))
    assert np.array_equal(nodes, oracle.nodes(g, sub, mode=oracle.MODE_FP32, node_step=node_step))
    orp, ovox, oln = oracle.rows(g, sub, mode=oracle.MODE_FP32, node_step=node_step)
    assert np.array_equal(rp, orp)
    assert np.array_equal(vox, ovox)
    err = np.abs(ln.astype(np.float64) - oln)
    assert np.all(err <= CHORD_TOL * np.maximum(oln, hmin)), err.max()
    return nodes


def _drop(pct, oracle, g, rec, n_blocks, n_sweeps, node_step=0.0):
    with pct.Context(g, n_blocks=n_blocks, node_step=node_step) as ctx:
        ctx.load(rec)
        ctx.iterate(n_sweeps)
        x = ctx.get_rsp().astype(np.float64)
    xo = oracle.drop(g, rec, n_blocks, n_sweeps, mode=oracle.MODE_FP32, node_step=node_step)
    err = np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)
    assert err.max() <= RSP_TOL, (err.max(), int(err.argmax()))


@pytest.mark.parametrize("step", [1.25, 3.0])
def test_rows_bit_exact_at_long_node_steps(pct, oracle, step):
    wl = S.head_workload(3000, seed=81)
    g = wl.grid
    rec = S.make_histories(wl)
    with pct.Context(g, n_blocks=2, node_step=step) as ctx:
        ctx.load(rec)
        nodes = _cmp_rows(oracle, g, rec, ctx, 0, 3000, node_step=step)
        _cmp_rows(oracle, g, rec, ctx, 1111, 257, node_step=step)  # a ragged interior range
    # the case under test happens: consecutive nodes more than a voxel apart on an axis
    span = np.abs(np.diff(nodes.reshape(3000, -1, 3).astype(np.int64), axis=1)).max()
    assert span > 2**20, span


@pytest.mark.parametrize("step", [1.25, 3.0])
def test_drop_parity_at_long_node_steps(pct, oracle, step):
    wl = S.head_workload(100_000, seed=82)
    _drop(pct, oracle, wl.grid, S.make_histories(wl), 5, 2, node_step=step)


def test_rows_bit_exact_on_the_anisotropic_grid(pct, oracle):
    g = W.training_grid()  # 200 x 200 x 48 of 1 x 1 x 2 mm
    wl = W.head_workload(g, 4000, seed=83)
    rec = S.make_histories(wl)
    for flags in (0, pct.FLAG_NO_SORT):
        with pct.Context(g, n_blocks=4, flags=flags) as ctx:
            ctx.load(rec)
            _cmp_rows(oracle, g, rec, ctx, 0, 4000)
            _cmp_rows(oracle, g, rec, ctx, 2049, 131)


def test_drop_parity_on_the_anisotropic_grid(pct, oracle):
    g = W.training_grid()
    wl = W.head_workload(g, 200_000, seed=84, n_blocks=50)
    _drop(pct, oracle, g, S.make_histories(wl), 50, 2)
