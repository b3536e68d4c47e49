"""pct_drop_block_noalloc: the entry point for callers that cannot allocate.

Some applications cannot allocate device memory once they are running (a
service that reserves all GPU memory for a fixed plan at start-up, a plugin
whose host owns every allocation). This entry point runs one DROP block update
on the caller's buffers using only a fixed scratch array inside the library.
The test calls it through the C ABI twice in a row and compares each result
with the context-based path (pct_iterate, one block, load order kept) and with
the FP64 oracle's one-block DROP, within the RSP tolerance of the parity
tests, for plain, uncompensated and clamped updates. The file sorts last so
that a run that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

RSP_TOL = 1e-3  # |x - x_ref| <= RSP_TOL * max(|x_ref|, 1), as in the parity tests


@pytest.fixture(scope="module")
def lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1707_05014_gb300 import build
    from paper_1707_05014_gb300 import pct as P

    build.build()
    L = P.load_library()
    L.pct_drop_block_noalloc.argtypes = [ctypes.POINTER(P._Grid), ctypes.POINTER(P._Config), ctypes.POINTER(P._Hist),
                                         ctypes.c_void_p, ctypes.c_void_p]
    L.pct_drop_block_noalloc.restype = ctypes.c_int
    return L


def _noalloc_call(L, P, g, rec_dev, x, lam=1.0, flags=0, clamp_min=0.0):
    import torch

    grid = P._Grid(g.nx, g.ny, g.nz, g.hx, g.hy, g.hz)
    cfg = P._Config(1, lam, 0.0, flags, clamp_min, 1, 128)
    h = P._Hist(len(rec_dev["t0"]), *[rec_dev[f].data_ptr() for f in P.FIELDS])
    stream = torch.cuda.current_stream().cuda_stream
    return L.pct_drop_block_noalloc(ctypes.byref(grid), ctypes.byref(cfg), ctypes.byref(h),
                                    ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("flags", [0, 2, 1], ids=["kahan", "no_kahan", "clamp"])
@pytest.mark.parametrize("kind,n", [("water", 20_000), ("head", 60_000)])
def test_noalloc_matches_context_path_on_two_calls(lib, oracle, kind, n, flags):
    import torch

    from paper_1707_05014_gb300 import pct as P

    wl = S.tiny_workload(n, seed=41) if kind == "water" else S.head_workload(n, seed=42)
    g = wl.grid
    rec = S.make_histories(wl)
    trec = {k: torch.from_numpy(v).cuda() for k, v in rec.items()}
    # the clamp floor sits above air so that the clamped update differs from the plain one
    clamp_min = 0.01 if flags & P.FLAG_CLAMP else 0.0

    # reference: the existing entry points, one block in load order, two sweeps
    refs = []
    with P.Context(g, n_blocks=1, flags=P.FLAG_NO_SORT | flags, clamp_min=clamp_min) as ctx:
        ctx.load(trec, borrow=True)
        for _ in range(2):
            ctx.iterate(1)
            refs.append(ctx.get_rsp().astype(np.float64))

    x = torch.zeros(g.m, dtype=torch.float32, device="cuda")
    for call in range(2):
        assert _noalloc_call(lib, P, g, trec, x, flags=flags, clamp_min=clamp_min) == 0, lib.pct_last_error()
        got = x.cpu().numpy().astype(np.float64)
        err = np.abs(got - refs[call]) / np.maximum(np.abs(refs[call]), 1.0)
        assert err.max() <= RSP_TOL, (call, err.max())
        assert np.abs(got).max() > 0
        if flags & P.FLAG_CLAMP:
            assert got.min() >= np.float32(clamp_min)
        # the oracle's DROP with one block, call + 1 sweeps (the FP32 node order)
        xo = oracle.drop(g, rec, 1, call + 1, mode=oracle.MODE_FP32,
                         clamp_min=clamp_min if flags & P.FLAG_CLAMP else None)
        err = np.abs(got - xo) / np.maximum(np.abs(xo), 1.0)
        assert err.max() <= RSP_TOL, (call, err.max())


def test_noalloc_rejects_grids_beyond_its_scratch(lib):
    import torch

    from paper_1707_05014_gb300 import pct as P

    g = S.Grid(200, 200, 64, 1.0, 1.0, 1.0)  # 2.56M voxels > 2,097,152
    rec = S.straight_records(g, [0.0], [0.0], [0.0], [0.0], [0.0])
    trec = {k: torch.from_numpy(v).cuda() for k, v in rec.items()}
    x = torch.zeros(g.m, dtype=torch.float32, device="cuda")
    assert _noalloc_call(lib, P, g, trec, x) == -5
    assert b"fixed scratch" in lib.pct_last_error()
    assert float(x.abs().max()) == 0.0
