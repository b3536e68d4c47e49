"""Batched persistent launch: several reconstructions of uneven size advance in
one launch per call (or as graph branches of per-block kernels, with one lane
or a group of lanes per history); each result equals its own context's pct_iterate and the
FP64 oracle's DROP (the same stages, Sec. 2.1 / Fig. 1) up to summation order,
element by element within the 0.1 % RSP bar, and a bounded wait
that cannot be met ends the launch with PCT_ERR_TIMEOUT instead of a hang."""
import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

RSP_TOL = 1e-3


@pytest.fixture(scope="module")
def P():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1707_05014_gb300 import build
    from paper_1707_05014_gb300 import pct

    build.build()
    return pct


def _workloads():
    return [
        (S.tiny_workload(30_000, seed=51), 3),
        (S.Workload("head_small", S.Grid(64, 64, 32, 3.125, 3.125, 3.125), 80_000, 52, 90, 100.0, 45.0, 7, 2, "head"), 7),
        (S.tiny_workload(7_001, seed=53), 1),
        (S.Workload("head80", S.Grid(80, 80, 40, 2.5, 2.5, 2.5), 50_000, 54, 45, 100.0, 45.0, 5, 2, "head"), 5),
    ]


@pytest.fixture(scope="module")
def oracle_images(oracle):
    """The FP64 oracle's DROP (FP32-order nodes) of every workload, 2 sweeps."""
    wls = _workloads()
    recs = [S.make_histories(w) for w, _ in wls]
    return recs, [oracle.drop(w.grid, r, B, 2, mode=oracle.MODE_FP32) for (w, B), r in zip(wls, recs)]


@pytest.mark.parametrize("mode,chunk,lanes", [(1, 0, 0), (1, 1000, 0), (2, 0, 0), (2, 0, 32), (2, 0, 8)])
def test_batch_matches_individual_contexts(P, oracle_images, mode, chunk, lanes):
    wls = _workloads()
    recs, oracle_x = oracle_images
    refs = []
    for (w, B), r in zip(wls, recs):
        with P.Context(w.grid, n_blocks=B) as c:
            c.load(r)
            c.iterate(2)
            refs.append(c.get_rsp().astype(np.float64))
    ctxs = []
    for (w, B), r in zip(wls, recs):
        c = P.Context(w.grid, n_blocks=B)
        c.load(r)
        ctxs.append(c)
    with P.Batch(ctxs, mode=mode, chunk=chunk, lanes=lanes) as b:
        b.iterate(1)
        b.iterate(1)
        b.sync()
        per_call = 1 if mode == 1 else sum(2 * B for _, B in wls)
        assert b.launches == 2 * per_call
    for c, ref, xo in zip(ctxs, refs, oracle_x):
        x = c.get_rsp().astype(np.float64)
        err = np.abs(x - ref) / np.maximum(np.abs(ref), 1.0)
        assert err.max() <= RSP_TOL, err.max()
        # and element-wise against the oracle's DROP of the same blocks
        err = np.abs(x - xo) / np.maximum(np.abs(xo), 1.0)
        assert err.max() <= RSP_TOL, err.max()
        c.close()


def test_batch_autotune_keeps_results(P):
    wls = _workloads()[:2]
    ctxs = []
    for w, B in wls:
        c = P.Context(w.grid, n_blocks=B)
        c.load(S.make_histories(w))
        ctxs.append(c)
    with P.Batch(ctxs) as b:
        choice = b.autotune()
        assert choice["mode"] in ("persistent", "graph_branches") and choice["sweep_ms"] > 0
        assert choice["lanes"] in (1, 16, 32)
        for c in ctxs:  # autotuning restores x
            assert float(np.abs(c.get_rsp()).max()) == 0.0
        b.iterate(1)
        b.sync()
    for c in ctxs:
        assert np.isfinite(c.get_rsp()).all()
        c.close()


def test_bounded_wait_reports_timeout_and_gpu_stays_usable(P):
    w, B = _workloads()[0]
    rec = S.make_histories(w)
    c = P.Context(w.grid, n_blocks=B)
    c.load(rec)
    with P.Batch([c], mode=P.BATCH_PERSISTENT, wait_limit_s=0.05, debug_unreachable_wait=True) as b:
        b.iterate(1)
        with pytest.raises(P.PctError) as ei:
            b.sync()
        assert ei.value.code == -6
    # the context and the GPU keep working
    with P.Batch([c], mode=P.BATCH_PERSISTENT) as b:
        b.iterate(1)
        b.sync()
    c.iterate(1)
    assert np.isfinite(c.get_rsp()).all()
    c.close()


def test_batch_refuses_a_reloaded_context(P):
    # the batch holds each context's records and block ranges as they were at
    # creation: after a reload (or a hull) it reports a state error, and a new
    # batch over the reloaded context runs
    w = S.tiny_workload(8000, seed=55)
    rec = S.make_histories(w)
    with P.Context(w.grid, n_blocks=2) as c:
        c.load(rec)
        with P.Batch([c]) as b:
            b.iterate(1)
            b.sync()
            c.load(S.subset(rec, slice(0, 5000)))
            with pytest.raises(P.PctError) as ei:
                b.iterate(1)
            assert ei.value.code == -7  # PCT_ERR_STATE
        with P.Batch([c]) as b:
            b.iterate(1)
            b.sync()
        assert np.isfinite(c.get_rsp()).all()
