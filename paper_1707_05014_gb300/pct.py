"""Thin Python binding of libpct (include/pct.h): argument marshalling only.

Every step of the reconstruction runs in the library's CUDA kernels; this
module only converts numpy arrays / torch tensors to pointers and status codes
to exceptions. PyTorch supplies device memory for caller-side buffers and the
current CUDA stream. If the compiled library is missing this module raises --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpct.so")

FIELDS = ("t0", "v0", "st0", "sv0", "t2", "v2", "st2", "sv2", "wepl", "cphi", "sphi")

PCT_OK = 0
STATUS = {
    -1: "INVALID_ARG", -2: "INVALID_DATA", -3: "NO_MEMORY", -4: "CUDA", -5: "CAPACITY", -6: "TIMEOUT", -7: "STATE",
}
FLAG_CLAMP = 1
FLAG_NO_KAHAN = 2
FLAG_PROFILE = 4
FLAG_NO_SORT = 8
FLAG_CARP = 16
LOAD_HOST = 0
LOAD_DEVICE_COPY = 1
LOAD_DEVICE_BORROW = 2


class PctError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pct {STATUS.get(code, code)}: {msg}")
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("hx", ctypes.c_double),
                ("hy", ctypes.c_double), ("hz", ctypes.c_double)]


class _Config(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int32), ("lam", ctypes.c_float), ("node_step_mm", ctypes.c_double),
                ("flags", ctypes.c_int32), ("clamp_min", ctypes.c_float), ("threads_per_proton", ctypes.c_int32),
                ("cta_threads", ctypes.c_int32), ("tvs_beta0", ctypes.c_float), ("tvs_alpha", ctypes.c_float),
                ("tvs_eps", ctypes.c_float), ("tvs_tries", ctypes.c_int32), ("carp_strings", ctypes.c_int32)]


class _Roofs(ctypes.Structure):
    _fields_ = [("l2_red_per_s", ctypes.c_double), ("l2_red_coherent_per_s", ctypes.c_double),
                ("l2_gather_per_s", ctypes.c_double), ("alu_ops_per_s", ctypes.c_double),
                ("fma_ops_per_s", ctypes.c_double), ("array_bytes", ctypes.c_int64), ("l2_bytes", ctypes.c_int64),
                ("sms", ctypes.c_int32)]


class _Hist(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(f, ctypes.c_void_p) for f in FIELDS]


_lib = None

_SIGS = {
    "pct_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_Grid), ctypes.POINTER(_Config), ctypes.c_int],
    "pct_destroy": [ctypes.c_void_p],
    "pct_set_stream": [ctypes.c_void_p, ctypes.c_void_p],
    "pct_geometry": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                     ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)],
    "pct_mlp_table": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "pct_load_histories": [ctypes.c_void_p, ctypes.POINTER(_Hist), ctypes.c_int, ctypes.POINTER(ctypes.c_int64)],
    "pct_mlp_rows": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)],
    "pct_block_counts": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p],
    "pct_block_weights": [ctypes.c_void_p],
    "pct_set_hull": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "pct_measure_roofs": [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p],
    "pct_carve_hull": [ctypes.c_void_p, ctypes.c_float, ctypes.c_int32],
    "pct_get_hull": [ctypes.c_void_p, ctypes.c_void_p],
    "pct_hull_ranges": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p],
    "pct_mlp_table_n": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p],
    "pct_project": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p],
    "pct_residual": [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)],
    "pct_set_x0": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "pct_iterate": [ctypes.c_void_p, ctypes.c_int32],
    "pct_get_rsp": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "pct_sync": [ctypes.c_void_p],
    "pct_last_sweep_times": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "pct_block_partial": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p],
    "pct_block_apply": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "pct_batch_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                         ctypes.c_void_p],
    "pct_batch_destroy": [ctypes.c_void_p],
    "pct_batch_iterate": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p],
    "pct_batch_sync": [ctypes.c_void_p, ctypes.c_void_p],
    "pct_batch_autotune": [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)],
    "pct_net_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                       ctypes.c_uint64, ctypes.c_int],
    "pct_net_destroy": [ctypes.c_void_p],
    "pct_net_get_params": [ctypes.c_void_p, ctypes.c_void_p],
    "pct_net_set_params": [ctypes.c_void_p, ctypes.c_void_p],
    "pct_net_forward": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "pct_net_gradients": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.POINTER(ctypes.c_double)],
    "pct_net_train_step": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float,
                           ctypes.POINTER(ctypes.c_double), ctypes.c_void_p],
    "pct_net_layer_shape": [ctypes.c_void_p, ctypes.c_int32] + [ctypes.POINTER(ctypes.c_int32)] * 4,
    "pct_net_layer": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 7,
}


def load_library(path: str = LIB_PATH):
    """Load libpct.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libpct.so not built at {path}: run paper_1707_05014_gb300.build.build()")
    L = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.pct_last_error.argtypes = []
    L.pct_last_error.restype = ctypes.c_char_p
    L.pct_launch_count.argtypes = [ctypes.c_void_p]
    L.pct_launch_count.restype = ctypes.c_int64
    L.pct_batch_launch_count.argtypes = [ctypes.c_void_p]
    L.pct_batch_launch_count.restype = ctypes.c_int64
    L.pct_net_param_count.argtypes = [ctypes.c_void_p]
    L.pct_net_param_count.restype = ctypes.c_int64
    L.pct_debug_fail_alloc.argtypes = [ctypes.c_int64]
    L.pct_debug_fail_alloc.restype = None
    if path == LIB_PATH:
        _lib = L
    return L


def _check(code: int):
    if code != PCT_OK:
        raise PctError(code, load_library().pct_last_error().decode())


def measure_roofs(device: int = 0, array_bytes: int = 8 << 20) -> Dict[str, float]:
    """The library's roof microbenchmarks (pct_measure_roofs) as a dict."""
    L = load_library()
    r = _Roofs()
    _check(L.pct_measure_roofs(int(device), int(array_bytes), ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in _Roofs._fields_}


def debug_fail_alloc(k: int) -> None:
    """Testing hook: the k-th device allocation of a context from now on fails
    (PCT_ERR_NO_MEMORY); k <= 0 disarms it."""
    load_library().pct_debug_fail_alloc(int(k))


def _torch():
    import torch

    return torch


def _check_vector(a, n: int, what: str, device: Optional[int] = None) -> None:
    """Raise ValueError unless `a` is a 1-D array or tensor of n values (and,
    for a CUDA tensor, on `device`): the library reads exactly n values from
    the pointer it is given."""
    shape = tuple(a.shape) if hasattr(a, "shape") else (len(a),)
    if len(shape) != 1 or shape[0] != n:
        raise ValueError(f"{what}: expected {n} values, got shape {shape}")
    if device is not None and _is_tensor(a) and a.is_cuda and a.device.index != device:
        raise ValueError(f"{what}: tensor on cuda:{a.device.index}, context on cuda:{device}")


def _is_tensor(a) -> bool:
    try:
        import torch

        return isinstance(a, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the handle of the legacy default stream


def _stream_ptr():
    """torch's current stream as a cudaStream_t; torch reports the legacy
    default stream as 0, which the C ABI reads as "the context's own stream",
    so it is passed as cudaStreamLegacy instead."""
    torch = _torch()
    h = torch.cuda.current_stream().cuda_stream
    return ctypes.c_void_p(h if h else CUDA_STREAM_LEGACY)


class Context:
    """One reconstruction: a grid, its MLP table, loaded histories and x.

    Mirrors pct_create / pct_load_histories / pct_mlp_rows / pct_iterate /
    pct_get_rsp. Device work runs on torch's current CUDA stream at the time of
    each call (pct_set_stream is refreshed before every call).
    """

    def __init__(self, grid, n_blocks: int = 10, lam: float = 1.0, node_step: float = 0.0, flags: int = 0,
                 clamp_min: float = 0.0, device: int = 0, cta_threads: int = 128, tvs_beta0: float = 0.0,
                 tvs_alpha: float = 0.99, tvs_eps: float = 1e-4, tvs_tries: int = 4, carp_strings: int = 0,
                 lanes: int = 1):
        L = load_library()
        self._L = L
        self.grid = grid
        self.lanes = int(lanes)
        g = _Grid(int(grid.nx), int(grid.ny), int(grid.nz), float(grid.hx), float(grid.hy), float(grid.hz))
        c = _Config(int(n_blocks), float(lam), float(node_step), int(flags), float(clamp_min), int(lanes),
                    int(cta_threads),
                    float(tvs_beta0), float(tvs_alpha), float(tvs_eps), int(tvs_tries), int(carp_strings))
        h = ctypes.c_void_p()
        _check(L.pct_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(c), int(device)))
        self._h = h
        self.device = device
        self.n_blocks = n_blocks
        self._keep = None
        R, du, K, E, M = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(L.pct_geometry(h, ctypes.byref(R), ctypes.byref(du), ctypes.byref(K), ctypes.byref(E), ctypes.byref(M)))
        self.R, self.du, self.K, self.E, self.M = R.value, du.value, K.value, E.value, M.value
        self.n = 0

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.pct_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _bind_stream(self):
        _check(self._L.pct_set_stream(self._h, _stream_ptr()))

    # -- calls -------------------------------------------------------------
    def mlp_table(self) -> np.ndarray:
        out = np.zeros((self.K + 1, 4), dtype=np.float64)
        self._bind_stream()
        _check(self._L.pct_mlp_table(self._h, out.ctypes.data_as(ctypes.c_void_p), 0))
        return out

    def load(self, rec: Dict, borrow: bool = False) -> None:
        """Load histories: numpy arrays (host copy) or CUDA tensors (device copy,
        or used in place with ``borrow=True``; the caller keeps them alive)."""
        arrs = [rec[f] for f in FIELDS]
        n = len(arrs[0])
        on_gpu = [_is_tensor(a) and a.is_cuda for a in arrs]
        for f, a in zip(FIELDS, arrs):
            _check_vector(a, n, f"history array {f!r}", self.device)
        if any(on_gpu) and not all(on_gpu):
            raise ValueError("history arrays must be all CUDA tensors or all host arrays")
        if on_gpu[0]:
            torch = _torch()
            arrs = [a.to(torch.float32).contiguous() for a in arrs]
            ptrs = [a.data_ptr() for a in arrs]
            flags = LOAD_DEVICE_BORROW if borrow else LOAD_DEVICE_COPY
        elif _is_tensor(arrs[0]):  # host tensors (e.g. pinned): copied by the library
            torch = _torch()
            arrs = [a.to(torch.float32).contiguous() for a in arrs]
            ptrs = [a.data_ptr() for a in arrs]
            flags = LOAD_HOST
        else:
            arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in arrs]
            ptrs = [a.ctypes.data for a in arrs]
            flags = LOAD_HOST
        h = _Hist(n, *ptrs)
        fb = ctypes.c_int64(-1)
        self._bind_stream()
        code = self._L.pct_load_histories(self._h, ctypes.byref(h), flags, ctypes.byref(fb))
        self.first_bad = fb.value
        _check(code)
        self._keep = arrs if flags == LOAD_DEVICE_BORROW else None
        self.n = n

    def rows(self, first: int = 0, count: Optional[int] = None, with_nodes: bool = False):
        """CSR rows of histories [first, first+count) as CUDA tensors:
        (row_ptr int64, vox int32, len float32[, nodes int32 (count, K+1, 3)])."""
        torch = _torch()
        count = self.n - first if count is None else count
        dev = torch.device("cuda", self.device)
        rp = torch.zeros(count + 1, dtype=torch.int64, device=dev)
        need = ctypes.c_int64(0)
        self._bind_stream()
        code = self._L.pct_mlp_rows(self._h, first, count, ctypes.c_void_p(rp.data_ptr()), None, None, 0, None,
                                    ctypes.byref(need))
        if code not in (PCT_OK, -5):
            _check(code)
        cap = max(int(need.value), 1)
        vox = torch.empty(cap, dtype=torch.int32, device=dev)
        ln = torch.empty(cap, dtype=torch.float32, device=dev)
        nodes = torch.empty((count, self.K + 1, 3), dtype=torch.int32, device=dev) if with_nodes else None
        _check(self._L.pct_mlp_rows(self._h, first, count, ctypes.c_void_p(rp.data_ptr()),
                                    ctypes.c_void_p(vox.data_ptr()), ctypes.c_void_p(ln.data_ptr()), cap,
                                    ctypes.c_void_p(nodes.data_ptr()) if nodes is not None else None,
                                    ctypes.byref(need)))
        n = int(need.value)
        out = (rp, vox[:n], ln[:n])
        return out + (nodes,) if with_nodes else out

    def set_hull(self, mask) -> None:
        """Object hull (M values, nonzero = inside; numpy or CUDA tensor), or
        None to remove it."""
        if mask is not None:
            if not _is_tensor(mask):
                mask = np.asarray(mask)
            _check_vector(mask.reshape(-1), self.M, "hull mask", self.device)
        self._bind_stream()
        if mask is None:
            _check(self._L.pct_set_hull(self._h, None, 0))
        elif _is_tensor(mask) and mask.is_cuda:
            m = (mask.reshape(-1) != 0).to(_torch().uint8).contiguous()
            _check(self._L.pct_set_hull(self._h, ctypes.c_void_p(m.data_ptr()), 1))
        else:
            m = np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0, dtype=np.uint8)
            _check(self._L.pct_set_hull(self._h, m.ctypes.data_as(ctypes.c_void_p), 0))

    def carve_hull(self, wepl_max: float, dilate: int = 1) -> None:
        """Space-carved hull from the loaded histories (see pct_carve_hull)."""
        self._bind_stream()
        _check(self._L.pct_carve_hull(self._h, float(wepl_max), int(dilate)))

    def get_hull(self) -> np.ndarray:
        out = np.zeros(self.M, dtype=np.uint8)
        self._bind_stream()
        _check(self._L.pct_get_hull(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def hull_ranges(self, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        """(count, 2) int32 hull entry/exit nodes of histories [first, first+count)."""
        count = self.n - first if count is None else count
        out = np.zeros((count, 2), dtype=np.int32)
        self._bind_stream()
        _check(self._L.pct_hull_ranges(self._h, int(first), int(count), out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def mlp_table_n(self, n: int) -> np.ndarray:
        """FP64 MLP table (n+1, 4) of a layer of n node intervals, from the GPU."""
        out = np.zeros((n + 1, 4), dtype=np.float64)
        self._bind_stream()
        _check(self._L.pct_mlp_table_n(self._h, int(n), out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def project(self, first: int = 0, count: Optional[int] = None):
        """a_i.x for histories [first, first+count) (load order) as a CUDA tensor."""
        torch = _torch()
        count = self.n - first if count is None else count
        y = torch.empty(count, dtype=torch.float32, device=torch.device("cuda", self.device))
        self._bind_stream()
        _check(self._L.pct_project(self._h, int(first), int(count), ctypes.c_void_p(y.data_ptr())))
        return y

    def residual(self, stride: int = 1) -> float:
        """sum (b_i - a_i.x)^2 over every stride-th stored history (synchronising)."""
        out = ctypes.c_double(0.0)
        self._bind_stream()
        _check(self._L.pct_residual(self._h, int(stride), ctypes.byref(out)))
        return out.value

    def block_counts(self, block: int):
        torch = _torch()
        out = torch.empty(self.M, dtype=torch.float32, device=torch.device("cuda", self.device))
        self._bind_stream()
        _check(self._L.pct_block_counts(self._h, int(block), ctypes.c_void_p(out.data_ptr())))
        return out

    def block_weights(self) -> None:
        """Form every block's DROP weights now (else the first sweep does)."""
        self._bind_stream()
        _check(self._L.pct_block_weights(self._h))

    def set_x0(self, x0) -> None:
        _check_vector(x0.reshape(-1) if hasattr(x0, "reshape") else x0, self.M, "x0", self.device)
        if _is_tensor(x0) and not x0.is_cuda:
            x0 = x0.numpy()
        self._bind_stream()
        if _is_tensor(x0):
            x0 = x0.to(_torch().float32).contiguous()
            _check(self._L.pct_set_x0(self._h, ctypes.c_void_p(x0.data_ptr()), 1))
            self._x0_keep = x0
        else:
            a = np.ascontiguousarray(np.asarray(x0).reshape(-1), dtype=np.float32)
            _check(self._L.pct_set_x0(self._h, a.ctypes.data_as(ctypes.c_void_p), 0))

    def iterate(self, n_sweeps: int) -> None:
        self._bind_stream()
        _check(self._L.pct_iterate(self._h, int(n_sweeps)))

    def get_rsp(self, device: bool = False):
        """x as a numpy array (synchronising) or a CUDA tensor (asynchronous)."""
        self._bind_stream()
        if device:
            torch = _torch()
            out = torch.empty(self.M, dtype=torch.float32, device=torch.device("cuda", self.device))
            _check(self._L.pct_get_rsp(self._h, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        out = np.empty(self.M, dtype=np.float32)
        _check(self._L.pct_get_rsp(self._h, out.ctypes.data_as(ctypes.c_void_p), 0))
        return out

    def last_sweep_times(self):
        """(fused_ms, apply_ms) per block of the most recent sweep (needs
        FLAG_PROFILE); synchronises."""
        f = np.zeros(self.n_blocks, dtype=np.float32)
        a = np.zeros(self.n_blocks, dtype=np.float32)
        self._bind_stream()
        _check(self._L.pct_last_sweep_times(self._h, f.ctypes.data_as(ctypes.c_void_p),
                                            a.ctypes.data_as(ctypes.c_void_p)))
        return f, a

    def block_partial(self, block: int, delta, counts=None) -> None:
        """This context's part of DROP block `block` (pct_block_partial) into the
        CUDA tensors delta (M floats) and, if given, counts (M floats)."""
        _check_vector(delta, self.M, "delta", self.device)
        if counts is not None:
            _check_vector(counts, self.M, "counts", self.device)
        self._bind_stream()
        _check(self._L.pct_block_partial(self._h, int(block), ctypes.c_void_p(delta.data_ptr()),
                                         ctypes.c_void_p(counts.data_ptr()) if counts is not None else None))

    def block_apply(self, delta, counts) -> None:
        """x += delta / counts where counts > 0 (pct_block_apply): the block
        update from sums over the ranks that share the block."""
        _check_vector(delta, self.M, "delta", self.device)
        _check_vector(counts, self.M, "counts", self.device)
        self._bind_stream()
        _check(self._L.pct_block_apply(self._h, ctypes.c_void_p(delta.data_ptr()), ctypes.c_void_p(counts.data_ptr())))

    def sync(self) -> None:
        self._bind_stream()
        _check(self._L.pct_sync(self._h))

    @property
    def launches(self) -> int:
        return int(self._L.pct_launch_count(self._h))


BATCH_PERSISTENT = 1
BATCH_GRAPH_BRANCHES = 2


class BatchConfig(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("branches", ctypes.c_int32), ("chunk", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("apply_tiles", ctypes.c_int32),
                ("wait_limit_s", ctypes.c_double), ("debug_unreachable_wait", ctypes.c_int32),
                ("lanes", ctypes.c_int32)]


class Batch:
    """Several loaded contexts advanced together by one persistent launch per
    call (pct_batch_*). The contexts must stay alive and loaded."""

    def __init__(self, contexts, mode: int = BATCH_GRAPH_BRANCHES, branches: int = 0, chunk: int = 0,
                 ctas_per_sm: int = 0, apply_tiles: int = 0, wait_limit_s: float = 0.0,
                 debug_unreachable_wait: bool = False, lanes: int = 0):
        L = load_library()
        self._L = L
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        self.cfg = BatchConfig(int(mode), int(branches), int(chunk), int(ctas_per_sm), int(apply_tiles),
                               float(wait_limit_s), 1 if debug_unreachable_wait else 0, int(lanes))
        h = ctypes.c_void_p()
        _check(L.pct_batch_create(ctypes.byref(h), arr, len(self.contexts), ctypes.byref(self.cfg)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.pct_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def iterate(self, n_sweeps: int) -> None:
        _check(self._L.pct_batch_iterate(self._h, int(n_sweeps), _stream_ptr()))

    def sync(self) -> None:
        _check(self._L.pct_batch_sync(self._h, _stream_ptr()))

    def autotune(self):
        chosen = BatchConfig()
        ms = ctypes.c_float(0.0)
        _check(self._L.pct_batch_autotune(self._h, ctypes.byref(chosen), ctypes.byref(ms)))
        return {"mode": "persistent" if chosen.mode == BATCH_PERSISTENT else "graph_branches",
                "branches": chosen.branches, "chunk": chosen.chunk, "ctas_per_sm": chosen.ctas_per_sm,
                "apply_tiles": chosen.apply_tiles, "lanes": chosen.lanes, "sweep_ms": ms.value}

    @property
    def launches(self) -> int:
        return int(self._L.pct_batch_launch_count(self._h))


NET_FORWARD, NET_DATA_GRAD, NET_WEIGHT_GRAD = 0, 1, 2


class Net:
    """Warm-start network (pct_net_*): x0 = x1 + f(x1) for nz x ny x nx volumes
    (CUDA float tensors in the reconstruction's voxel order)."""

    def __init__(self, nz: int, ny: int, nx: int, seed: int = 0, device: int = 0):
        L = load_library()
        self._L = L
        self.shape = (nz, ny, nx)
        self.device = device
        h = ctypes.c_void_p()
        _check(L.pct_net_create(ctypes.byref(h), int(nz), int(ny), int(nx), int(seed), int(device)))
        self._h = h
        self.n_params = int(L.pct_net_param_count(h))
        self._scratch = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.pct_net_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _volume(self, t, what: str):
        """t as a contiguous float32 CUDA tensor of nz*ny*nx values on the
        network's device (the library reads exactly that many)."""
        m = self.shape[0] * self.shape[1] * self.shape[2]
        if not (_is_tensor(t) and t.is_cuda):
            raise ValueError(f"{what}: expected a CUDA tensor")
        _check_vector(t.reshape(-1), m, what, self.device)
        return t.to(_torch().float32).contiguous()

    def _x0(self):
        torch = _torch()
        if self._scratch is None:
            n = self.shape[0] * self.shape[1] * self.shape[2]
            self._scratch = torch.empty(n, dtype=torch.float32, device=torch.device("cuda", self.device))
        return self._scratch

    def layer_shape(self, layer: int):
        """(Cin, Cout, input level, output level) of a layer."""
        v = [ctypes.c_int32() for _ in range(4)]
        _check(self._L.pct_net_layer_shape(self._h, int(layer), *[ctypes.byref(x) for x in v]))
        return tuple(int(x.value) for x in v)

    def layer(self, layer: int, op: int, inp=None, skip=None, dy=None, mask=None, add=None):
        """One layer through pct_net_layer. BF16 operands are int16 CUDA
        tensors of bit patterns, channels last; returns the output as an int16
        (BF16 bits) tensor, or float32 for NET_WEIGHT_GRAD (dW then db).
        Synchronises."""
        torch = _torch()
        cin, cout, lin, lout = self.layer_shape(layer)
        nz, ny, nx = self.shape
        vox = lambda lv: (nz >> lv) * (ny >> lv) * (nx >> lv)  # noqa: E731
        dev = torch.device("cuda", self.device)
        want = {"inp": (inp, vox(lin) * cin), "skip": (skip, vox(lout) * cout), "dy": (dy, vox(lout) * cout),
                "mask": (mask, vox(lin) * cin), "add": (add, vox(lin) * cin)}
        ptr = {}
        keep = []
        for name, (t, n) in want.items():
            if t is None:
                ptr[name] = None
                continue
            if not (_is_tensor(t) and t.is_cuda and t.dtype == torch.int16):
                raise ValueError(f"{name}: expected an int16 CUDA tensor of BF16 bit patterns")
            _check_vector(t.reshape(-1), n, name, self.device)
            t = t.contiguous()
            keep.append(t)
            ptr[name] = ctypes.c_void_p(t.data_ptr())
        if op == NET_FORWARD:
            out = torch.empty(vox(lout) * cout, dtype=torch.int16, device=dev)
        elif op == NET_DATA_GRAD:
            out = torch.empty(vox(lin) * cin, dtype=torch.int16, device=dev)
        else:
            out = torch.empty(27 * cin * cout + cout, dtype=torch.float32, device=dev)
        _check(self._L.pct_net_layer(self._h, int(layer), int(op), ptr["inp"], ptr["skip"], ptr["dy"], ptr["mask"],
                                     ptr["add"], ctypes.c_void_p(out.data_ptr()), _stream_ptr()))
        torch.cuda.synchronize(dev)
        return out

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(self._L.pct_net_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, p: np.ndarray) -> None:
        a = np.ascontiguousarray(p, dtype=np.float32)
        _check_vector(a.reshape(-1), self.n_params, "network parameters")
        _check(self._L.pct_net_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p)))

    def forward(self, x1):
        torch = _torch()
        x1 = self._volume(x1, "x1")
        x0 = torch.empty_like(x1)
        _check(self._L.pct_net_forward(self._h, ctypes.c_void_p(x1.data_ptr()), ctypes.c_void_p(x0.data_ptr()),
                                       _stream_ptr()))
        return x0

    def gradients(self, x1, target):
        torch = _torch()
        x1 = self._volume(x1, "x1")
        target = self._volume(target, "target")
        torch.cuda.synchronize()
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(self._L.pct_net_gradients(self._h, ctypes.c_void_p(x1.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                         ctypes.c_void_p(self._x0().data_ptr()), g.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(loss)))
        return loss.value, g

    def train_step(self, x1, target, lr: float = 1e-3, want_loss: bool = True):
        x1 = self._volume(x1, "x1")
        target = self._volume(target, "target")
        loss = ctypes.c_double(0.0)
        _check(self._L.pct_net_train_step(self._h, ctypes.c_void_p(x1.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                          ctypes.c_void_p(self._x0().data_ptr()), float(lr),
                                          ctypes.byref(loss) if want_loss else None, _stream_ptr()))
        return loss.value if want_loss else None
