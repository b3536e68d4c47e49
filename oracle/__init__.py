"""FP64 CPU oracle for the proton-CT hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package. It wraps ``pct_oracle.c`` (plain C,
FP64, single-threaded except ``drop_threads``) through ctypes; it shares no
code with the CUDA library.

Functions (all follow arXiv 1707.05014 Sec. 2 / 2.1 and the MLP form of
Schulte et al. 2008 that Sec. 2 cites):

* ``mlp_table``   -- per-node coefficients (c1, c2, c3, c4), Sec. 2 (MLP).
* ``mlp_table_n`` -- the same for a water layer of n node intervals (object hull).
* ``nodes``       -- quantised interior MLP nodes (FP64 or FP32-mirror order).
* ``rows``        -- CSR rows of A: voxel indices and chord lengths, Sec. 2.
* ``reentries``   -- how often a row re-enters a voxel (where run counts and the
  textbook one-entry-per-voxel row differ).
* ``project``     -- a_i . x for a range of protons.
* ``block_counts``-- s_j of one DROP block.
* ``drop``        -- DROP sweeps, Sec. 2.1 / Fig. 1.
* ``drop_threads``-- the same sweeps with each block split over OpenMP threads
  (sums in another order; used to time the oracle on all host cores).
* ``carp``        -- CARP sweeps, Sec. 2.2 / Fig. 2 (strings + component averaging).
* ``solve_tvs``   -- DROP / CARP with total-variation superiorization, Sec. 4.2.
* ``hull_ranges``, ``carve_hull`` -- MLP inside an object hull: per-history
  hull entry/exit nodes, and the hull carved from low-WEPL histories.

Pins (tests/test_oracle_*.py): the energy polynomial against the relativistic
entry value and a Bethe-stopping integration in water, table identities
(translation / straight-line invariance, depth reversal), the
constant-scattering special case against the cubic Hermite interpolant, the
table against the Gaussian-conditioning form, quadrature against closed-form
polynomial integrals, straight-line and tie-rule walks, brute-force
supersampled chords, total chord = clipped polyline length, DROP against a
dense weighted least-squares solve and the one-row ART projection, hull layer
tables, ranges and carving against independent re-derivations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pct_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

MODE_FP64 = 0
MODE_FP32 = 1
F_CONST_SCATTER = 1
F_NO_LOG = 2

FIELDS = ("t0", "v0", "st0", "sv0", "t2", "v2", "st2", "sv2", "wepl", "cphi", "sphi")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                               "-shared", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("hx", ctypes.c_double),
                ("hy", ctypes.c_double), ("hz", ctypes.c_double), ("node_step", ctypes.c_double),
                ("hull", ctypes.POINTER(ctypes.c_uint8))]


class _Rec(ctypes.Structure):
    _fields_ = [(f, ctypes.POINTER(ctypes.c_float)) for f in FIELDS]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        dp = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        gp = ctypes.POINTER(_Grid)
        rp = ctypes.POINTER(_Rec)
        L.or_geom_info.argtypes = [gp, dp, dp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.or_inv_beta2p2.argtypes = [ctypes.c_double, ctypes.c_int]
        L.or_inv_beta2p2.restype = ctypes.c_double
        L.or_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
        L.or_moment.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        L.or_moment.restype = ctypes.c_double
        L.or_scatter_cov.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
        L.or_scatter_cov.restype = None
        L.or_mlp_table.argtypes = [gp, ctypes.c_int, dp]
        L.or_mlp_table_n.argtypes = [gp, ctypes.c_int, ctypes.c_int, dp]
        L.or_hull_ranges.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, i32p]
        L.or_carve_hull.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_uint8)]
        L.or_nodes.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, i32p]
        L.or_polyline.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_int, i32p]
        L.or_rows.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, i64p, i32p, dp,
                              ctypes.c_int64]
        L.or_rows.restype = ctypes.c_int64
        L.or_project.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, dp, dp]
        L.or_block_counts.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.or_tv_value.argtypes = [gp, dp, ctypes.c_double]
        L.or_tv_value.restype = ctypes.c_double
        L.or_tv_grad.argtypes = [gp, dp, ctypes.c_double, dp]
        L.or_solve_tvs.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, dp]
        L.or_carp.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                              ctypes.c_int, dp, dp]
        L.or_drop.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, ctypes.c_double, dp, dp]
        L.or_drop_threads.argtypes = [gp, dp, rp, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, dp, dp]
        L.or_max_threads.argtypes = []
        L.or_max_threads.restype = ctypes.c_int
    return _lib


def _grid(g, node_step: float = 0.0, hull=None) -> _Grid:
    """C grid descriptor; ``hull`` (M values, nonzero = inside the object) is
    kept alive on the returned structure."""
    gg = _Grid(int(g.nx), int(g.ny), int(g.nz), float(g.hx), float(g.hy), float(g.hz), float(node_step), None)
    if hull is not None:
        h = np.ascontiguousarray(np.asarray(hull).reshape(-1) != 0, dtype=np.uint8)
        if h.size != g.nx * g.ny * g.nz:
            raise ValueError("hull mask must hold one value per voxel")
        gg.hull = h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        gg._keep = h
    return gg


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class _RecHolder:
    def __init__(self, rec: Dict[str, np.ndarray]):
        self.arrs = {f: np.ascontiguousarray(rec[f], dtype=np.float32) for f in FIELDS}
        self.n = len(self.arrs["t0"])
        self.s = _Rec(*[_ptr(self.arrs[f], ctypes.c_float) for f in FIELDS])


def geom_info(g, node_step: float = 0.0) -> Tuple[float, float, int, int]:
    """(R, du, K, E): plane half-distance, node spacing, interior node count - 1,
    extension nodes per side."""
    R = ctypes.c_double()
    du = ctypes.c_double()
    K = ctypes.c_int()
    E = ctypes.c_int()
    gg = _grid(g, node_step)
    lib().or_geom_info(ctypes.byref(gg), ctypes.byref(R), ctypes.byref(du), ctypes.byref(K), ctypes.byref(E))
    return R.value, du.value, K.value, E.value


def inv_beta2p2(w_cm: float, flags: int = 0) -> float:
    return lib().or_inv_beta2p2(float(w_cm), int(flags))


def scatter_cov(a_cm: float, b_cm: float, flags: int = 0) -> np.ndarray:
    """Scattering covariance (position-position, position-slope, slope-slope)
    of the water slab between depths a and b (cm), the building block of the
    MLP matrices."""
    out = np.zeros(3)
    lib().or_scatter_cov(ctypes.c_double(a_cm), ctypes.c_double(b_cm), ctypes.c_int(flags),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def gauss_legendre(n: int) -> Tuple[np.ndarray, np.ndarray]:
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss_legendre(n, _ptr(x, ctypes.c_double), _ptr(w, ctypes.c_double))
    return x, w


def moment(a: float, b: float, c: float, m: int, flags: int = 0) -> float:
    return lib().or_moment(float(a), float(b), float(c), int(m), int(flags))


def mlp_table(g, flags: int = 0, node_step: float = 0.0) -> np.ndarray:
    """(K+1, 4) float64: c1, c2 [mm], c3, c4 [mm] per interior node."""
    _, _, K, _ = geom_info(g, node_step)
    out = np.zeros((K + 1, 4))
    gg = _grid(g, node_step)
    lib().or_mlp_table(ctypes.byref(gg), int(flags), _ptr(out, ctypes.c_double))
    return out


def mlp_table_n(g, n: int, flags: int = 0, node_step: float = 0.0) -> np.ndarray:
    """(n+1, 4) float64: the MLP table of a hull n node intervals thick (nodes
    m = 0..n from the hull entry); n = K is the slab between the planes."""
    out = np.zeros((n + 1, 4))
    gg = _grid(g, node_step)
    if lib().or_mlp_table_n(ctypes.byref(gg), int(flags), int(n), _ptr(out, ctypes.c_double)) != n:
        raise ValueError("n outside [1, K]")
    return out


def hull_ranges(g, rec, hull, first: int = 0, count: Optional[int] = None, mode: int = MODE_FP32,
                node_step: float = 0.0) -> np.ndarray:
    """(count, 2) int32: hull entry and exit node of each proton ((0, K) for a
    proton that misses the hull)."""
    h = _RecHolder(rec)
    count = h.n - first if count is None else count
    tab = _tab(g, None, 0, node_step)
    out = np.zeros((count, 2), dtype=np.int32)
    gg = _grid(g, node_step, hull)
    lib().or_hull_ranges(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), first, count, mode,
                         _ptr(out, ctypes.c_int32))
    return out


def carve_hull(g, rec, wepl_max: float, dilate: int = 0, mode: int = MODE_FP32, node_step: float = 0.0) -> np.ndarray:
    """Space-carved hull (M uint8): voxels on the rows of protons with WEPL <=
    wepl_max are outside; the rest, grown by ``dilate`` 6-neighbour steps, is
    the hull."""
    h = _RecHolder(rec)
    tab = _tab(g, None, 0, node_step)
    out = np.zeros(g.nx * g.ny * g.nz, dtype=np.uint8)
    gg = _grid(g, node_step)
    lib().or_carve_hull(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), h.n, float(wepl_max),
                        int(dilate), mode, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return out


def _tab(g, table, flags, node_step):
    if table is None:
        table = mlp_table(g, flags, node_step)
    return np.ascontiguousarray(table, dtype=np.float64)


def nodes(g, rec, first: int = 0, count: Optional[int] = None, mode: int = MODE_FP32, table=None, flags: int = 0,
          node_step: float = 0.0, hull=None) -> np.ndarray:
    """(count, K+1, 3) int32 Q20 grid coordinates of the interior nodes."""
    h = _RecHolder(rec)
    count = h.n - first if count is None else count
    tab = _tab(g, table, flags, node_step)
    out = np.zeros((count, tab.shape[0], 3), dtype=np.int32)
    gg = _grid(g, node_step, hull)
    lib().or_nodes(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), first, count, mode,
                   _ptr(out, ctypes.c_int32))
    return out


def polyline(g, rec, i: int, mode: int = MODE_FP32, table=None, flags: int = 0, node_step: float = 0.0, hull=None):
    """(K + 2E + 1, 3) int32 Q20 nodes of proton i, extensions included."""
    h = _RecHolder(rec)
    tab = _tab(g, table, flags, node_step)
    _, _, K, E = geom_info(g, node_step)
    out = np.zeros((K + 2 * E + 1, 3), dtype=np.int32)
    gg = _grid(g, node_step, hull)
    lib().or_polyline(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), int(i), mode,
                      _ptr(out, ctypes.c_int32))
    return out


def rows(g, rec, first: int = 0, count: Optional[int] = None, mode: int = MODE_FP32, table=None, flags: int = 0,
         node_step: float = 0.0, hull=None):
    """CSR rows: (row_ptr int64 [count+1], vox int32, len float64 mm)."""
    h = _RecHolder(rec)
    count = h.n - first if count is None else count
    tab = _tab(g, table, flags, node_step)
    gg = _grid(g, node_step, hull)
    rp = np.zeros(count + 1, dtype=np.int64)
    cap = max(1, 64 * count)
    while True:
        vox = np.zeros(cap, dtype=np.int32)
        ln = np.zeros(cap, dtype=np.float64)
        need = lib().or_rows(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), first, count, mode,
                             _ptr(rp, ctypes.c_int64), _ptr(vox, ctypes.c_int32), _ptr(ln, ctypes.c_double), cap)
        if need <= cap:
            return rp, vox[:need].copy(), ln[:need].copy()
        cap = int(need)


def reentries(g, rec, first: int = 0, count: Optional[int] = None, mode: int = MODE_FP32, node_step: float = 0.0,
              hull=None) -> Dict[str, int]:
    """How often a row returns to a voxel it has already left (Sec. 2 rows).

    Runs are maximal stretches in one voxel, and the convention here counts
    runs: s_j = runs in voxel j over a block, |a_i|^2 = sum of squared run
    lengths. Both equal the textbook row (one entry per voxel) exactly when no
    row re-enters a voxel; this reports how often one does. Returns the number
    of rows, of rows with a re-entered voxel, of runs, and of runs beyond the
    first in their voxel."""
    rp, vox, _ = rows(g, rec, first, count, mode=mode, node_step=node_step, hull=hull)
    n = len(rp) - 1
    M = int(g.nx) * int(g.ny) * int(g.nz)
    row = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    keys = np.unique(row * M + vox.astype(np.int64))
    distinct = np.bincount(keys // M, minlength=n)
    return {"rows": n, "rows_with_reentry": int(np.count_nonzero(distinct < np.diff(rp))),
            "runs": int(len(vox)), "repeated_runs": int(len(vox) - len(keys))}


def project(g, rec, x: np.ndarray, first: int = 0, count: Optional[int] = None, mode: int = MODE_FP32, table=None,
            flags: int = 0, node_step: float = 0.0, hull=None) -> np.ndarray:
    h = _RecHolder(rec)
    count = h.n - first if count is None else count
    tab = _tab(g, table, flags, node_step)
    gg = _grid(g, node_step, hull)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(count)
    lib().or_project(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), first, count, mode,
                     _ptr(xx, ctypes.c_double), _ptr(y, ctypes.c_double))
    return y


def block_counts(g, rec, n_blocks: int, b: int, mode: int = MODE_FP32, table=None, flags: int = 0,
                 node_step: float = 0.0, hull=None) -> np.ndarray:
    h = _RecHolder(rec)
    tab = _tab(g, table, flags, node_step)
    gg = _grid(g, node_step, hull)
    out = np.zeros(g.nx * g.ny * g.nz)
    lib().or_block_counts(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), h.n, n_blocks, b, mode,
                          _ptr(out, ctypes.c_double))
    return out


def drop(g, rec, n_blocks: int, n_sweeps: int, lam: float = 1.0, x0: Optional[np.ndarray] = None,
         mode: int = MODE_FP32, table=None, flags: int = 0, node_step: float = 0.0, hull=None, clamp_min: Optional[float] = None,
         return_resid: bool = False):
    """DROP reconstruction (Sec. 2.1). Returns x (float64, M)."""
    h = _RecHolder(rec)
    tab = _tab(g, table, flags, node_step)
    gg = _grid(g, node_step, hull)
    M = g.nx * g.ny * g.nz
    x = np.zeros(M) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    resid = np.zeros(max(n_sweeps, 1))
    rc = lib().or_drop(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), h.n, n_blocks, float(lam),
                       n_sweeps, mode, clamp_min is not None, float(clamp_min or 0.0), _ptr(x, ctypes.c_double),
                       _ptr(resid, ctypes.c_double))
    if rc != 0:
        raise MemoryError("oracle drop: allocation failed")
    return (x, resid[:n_sweeps]) if return_resid else x


def drop_threads(g, rec, n_blocks: int, n_sweeps: int, threads: int = 0, lam: float = 1.0,
                 x0: Optional[np.ndarray] = None, mode: int = MODE_FP32, node_step: float = 0.0, hull=None):
    """DROP as ``drop`` with each block's histories split over ``threads``
    OpenMP threads (0: all); only the order of the sums differs."""
    h = _RecHolder(rec)
    tab = _tab(g, None, 0, node_step)
    gg = _grid(g, node_step, hull)
    M = g.nx * g.ny * g.nz
    x = np.zeros(M) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    resid = np.zeros(max(n_sweeps, 1))
    rc = lib().or_drop_threads(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), h.n, n_blocks,
                               float(lam), n_sweeps, mode, int(threads), _ptr(x, ctypes.c_double),
                               _ptr(resid, ctypes.c_double))
    if rc != 0:
        raise MemoryError("oracle drop_threads: allocation failed")
    return x


def max_threads() -> int:
    return int(lib().or_max_threads())


def carp(g, rec, n_strings: int, n_sweeps: int, lam: float = 1.0, x0: Optional[np.ndarray] = None,
         mode: int = MODE_FP32, table=None, flags: int = 0, node_step: float = 0.0, hull=None, return_resid: bool = False,
         n_blocks: Optional[int] = None):
    """CARP reconstruction (Sec. 2.2): strings of consecutive DROP blocks
    (n_blocks, default one block per string) swept from a common x0, then
    component averaging. Returns x (float64, M)."""
    n_blocks = n_strings if n_blocks is None else n_blocks
    h = _RecHolder(rec)
    tab = _tab(g, table, flags, node_step)
    gg = _grid(g, node_step, hull)
    M = g.nx * g.ny * g.nz
    x = np.zeros(M) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    resid = np.zeros(max(n_sweeps, 1))
    rc = lib().or_carp(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), h.n, n_blocks, n_strings,
                       float(lam), n_sweeps, mode, _ptr(x, ctypes.c_double), _ptr(resid, ctypes.c_double))
    if rc != 0:
        raise MemoryError("oracle carp: allocation failed")
    return (x, resid[:n_sweeps]) if return_resid else x


def tv_value(g, x: np.ndarray, eps: float = 1e-4) -> float:
    """TV_eps of an image (forward differences, Neumann far boundary)."""
    xx = np.ascontiguousarray(x, dtype=np.float64)
    gg = _grid(g)
    return lib().or_tv_value(ctypes.byref(gg), _ptr(xx, ctypes.c_double), float(eps))


def tv_grad(g, x: np.ndarray, eps: float = 1e-4) -> np.ndarray:
    xx = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(xx)
    gg = _grid(g)
    lib().or_tv_grad(ctypes.byref(gg), _ptr(xx, ctypes.c_double), float(eps), _ptr(out, ctypes.c_double))
    return out


def solve_tvs(g, rec, n_blocks: int, n_sweeps: int, lam: float = 1.0, carp: int = 0, beta0: float = 0.02,
              alpha: float = 0.99, eps: float = 1e-4, tries: int = 4, x0: Optional[np.ndarray] = None,
              mode: int = MODE_FP32, table=None, flags: int = 0, node_step: float = 0.0, hull=None) -> np.ndarray:
    """DROP (TVS before every block) or, with carp = number of strings > 0,
    CARP (TVS before every iteration), with total-variation superiorization
    (Sec. 4.2)."""
    h = _RecHolder(rec)
    tab = _tab(g, table, flags, node_step)
    gg = _grid(g, node_step, hull)
    M = g.nx * g.ny * g.nz
    x = np.zeros(M) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rc = lib().or_solve_tvs(ctypes.byref(gg), _ptr(tab, ctypes.c_double), ctypes.byref(h.s), h.n, n_blocks,
                            float(lam), n_sweeps, mode, int(carp), float(beta0), float(alpha), float(eps),
                            int(tries), _ptr(x, ctypes.c_double))
    if rc != 0:
        raise MemoryError("oracle tvs: allocation failed")
    return x
