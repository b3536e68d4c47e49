"""Host-side argument checks of the Python binding: arrays whose length does
not match what the library will read are refused before any library call
(the library reads exactly n record values and M voxel values from the
pointers it is given)."""
import ctypes

import numpy as np
import pytest

from paper_1707_05014_gb300 import pct
from paper_1707_05014_gb300 import synthetic as S


class _NoLibrary:
    """Stands in for libpct: any call means a check let bad input through."""

    def __getattr__(self, name):
        raise AssertionError(f"{name} called with arguments the binding should have refused")


def _context(M=1000):
    ctx = pct.Context.__new__(pct.Context)
    ctx._L = _NoLibrary()
    ctx._h = ctypes.c_void_p()
    ctx.device = 0
    ctx.M = M
    ctx.n = 0
    return ctx


def test_load_refuses_arrays_of_unequal_length():
    rec = S.make_histories(S.tiny_workload(100, seed=1))
    rec["wepl"] = rec["wepl"][:99]
    with pytest.raises(ValueError, match="wepl"):
        _context().load(rec)


def test_load_refuses_two_dimensional_arrays():
    rec = S.make_histories(S.tiny_workload(100, seed=1))
    rec["st2"] = rec["st2"].reshape(10, 10)
    with pytest.raises(ValueError, match="st2"):
        _context().load(rec)


def test_load_refuses_mixed_host_and_device_arrays():
    torch = pytest.importorskip("torch")
    rec = S.make_histories(S.tiny_workload(100, seed=1))
    rec["t0"] = torch.from_numpy(rec["t0"])
    ctx = _context()

    class FakeCuda:  # a CUDA-looking tensor: is_cuda, same length, on cuda:0
        is_cuda = True
        shape = (100,)
        device = type("D", (), {"index": 0})()

    rec["v0"] = FakeCuda()
    pct_is_tensor = pct._is_tensor
    try:
        pct._is_tensor = lambda a: isinstance(a, (torch.Tensor, FakeCuda))
        with pytest.raises(ValueError, match="all CUDA tensors or all host"):
            ctx.load(rec)
    finally:
        pct._is_tensor = pct_is_tensor


def test_x0_and_hull_must_hold_one_value_per_voxel():
    ctx = _context(M=1000)
    with pytest.raises(ValueError, match="x0"):
        ctx.set_x0(np.zeros(999, np.float32))
    with pytest.raises(ValueError, match="x0"):
        ctx.set_x0([0.0] * 1001)
    with pytest.raises(ValueError, match="hull mask"):
        ctx.set_hull(np.ones(1001, np.uint8))
    with pytest.raises(ValueError, match="hull mask"):
        ctx.set_hull(np.ones((10, 10, 9), np.uint8))


def test_network_volumes_must_match_its_grid():
    net = pct.Net.__new__(pct.Net)
    net._L = _NoLibrary()
    net._h = ctypes.c_void_p()
    net.shape = (4, 5, 6)
    net.device = 0
    with pytest.raises(ValueError, match="CUDA tensor"):
        net.forward(np.zeros(120, np.float32))
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError, match="CUDA tensor"):
        net.train_step(torch.zeros(120), torch.zeros(120))
    net.n_params = 10
    with pytest.raises(ValueError, match="network parameters"):
        net.set_params(np.zeros(9, np.float32))
