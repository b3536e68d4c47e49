"""The first DROP sweep after a load forms the block weights s_j (Sec. 2.1) as it
goes. With one lane per history and no hull, CARP or TVS it adds (a_ij r_i, 1)
per run to a float pair by one vector reduction; a float count is exact below
2^24, and where one voxel collects 2^24 or more runs of one block the sweep is
undone and done again with integer counts. Either way the image equals the
one from weights formed ahead with integer counts (pct_block_weights), within
the float summation order, and the counts are exact.

The grid is one voxel of 2 mm crossed by straight paths, so the block count
of that voxel is the number of histories: 1M stays on the float path, 17M
(above 2^24 = 16,777,216) takes the integer redo."""
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


def _straight_through_one_voxel(g, n, seed):
    rng = np.random.Generator(np.random.Philox(seed))
    rec = S.straight_records(g, rng.uniform(-0.8, 0.8, n), rng.uniform(-0.8, 0.8, n), np.zeros(n), np.zeros(n),
                             rng.uniform(0.0, 2.0 * np.pi, n))
    rec["wepl"] = rng.uniform(1.5, 2.5, n).astype(np.float32)
    return rec


@pytest.mark.parametrize("n, redo", [(1_000_000, False), (17_000_000, True)], ids=["float_counts", "integer_redo"])
def test_first_sweep_weights_match_integer_weights(pct, n, redo):
    g = S.Grid(1, 1, 1, 2.0, 2.0, 2.0)
    rec = _straight_through_one_voxel(g, n, seed=64)
    with pct.Context(g, n_blocks=1) as a:
        a.load(rec)
        before = a.launches
        a.iterate(1)
        x = a.get_rsp().astype(np.float64)
        used = a.launches - before
        counts = a.block_counts(0).cpu().numpy()
    with pct.Context(g, n_blocks=1) as b:
        b.load(rec)
        b.block_weights()
        b.iterate(1)
        y = b.get_rsp().astype(np.float64)
    assert counts[0] == n  # every path crosses the voxel once
    # one sweep of one block is two launches; the redo adds the integer
    # weights (two launches) and the sweep again
    assert used == (6 if redo else 2)
    # one float accumulator per voxel takes all n updates in an order set by
    # the atomics: the parity bar of the images, 1e-3 relative
    assert y[0] > 0 and abs(x[0] - y[0]) <= 1e-3 * y[0]
