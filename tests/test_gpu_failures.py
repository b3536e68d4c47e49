"""Allocation failure, injected on the host (pct_debug_fail_alloc makes the k-th
device allocation of a context fail as if the device were out of memory): every
failing call reports PCT_ERR_NO_MEMORY, frees what it had allocated, and the
context stays usable."""
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
    yield P
    P.debug_fail_alloc(0)


def test_create_reports_every_failing_allocation_and_frees_the_rest(pct):
    import torch

    g = S.Grid(64, 64, 64, 1.0, 1.0, 1.0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(1, 8):  # a plain DROP context makes seven device allocations
        pct.debug_fail_alloc(k)
        with pytest.raises(pct.PctError) as ei:
            pct.Context(g, n_blocks=2)
        assert ei.value.code == -3, k
    pct.debug_fail_alloc(0)
    with pct.Context(g, n_blocks=2):  # the eighth would not fail: creation works again
        pass
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 16 << 20


@pytest.mark.parametrize("k", [1, 2, 3])
def test_failed_load_leaves_a_usable_context(pct, oracle, k):
    wl = S.tiny_workload(6000, seed=94)
    rec = S.make_histories(wl)
    with pct.Context(wl.grid, n_blocks=3) as ctx:
        pct.debug_fail_alloc(k)
        with pytest.raises(pct.PctError) as ei:
            ctx.load(rec)
        assert ei.value.code == -3
        pct.debug_fail_alloc(0)
        with pytest.raises(pct.PctError) as ei:
            ctx.iterate(1)  # nothing is loaded after the failure
        assert ei.value.code == -7
        ctx.load(rec)
        ctx.iterate(2)
        x = ctx.get_rsp().astype(np.float64)
    xo = oracle.drop(wl.grid, rec, 3, 2, mode=oracle.MODE_FP32)
    assert np.max(np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)) <= 1e-3
