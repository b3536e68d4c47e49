"""Seeded synthetic proton histories and phantoms (input generation only).

This module makes the inputs that both the CUDA path and the oracle consume. It
holds none of the reconstruction's arithmetic: no most-likely path, no voxel
walk, no projection update. What it does compute is the *scanner stand-in*:

* a phantom (an additive set of axis-aligned ellipsoids / z-cylinders on an air
  background) and its voxelised RSP image ``x_true``;
* per-proton entry/exit states at the two measurement planes, with a simple
  Gaussian multiple-scattering spread of the exit state (a fixed recipe of this
  generator, not the reconstruction's MLP model);
* the WEPL of each proton as the straight entry->exit chord's RSP line integral
  (analytic line/quadric intersections), times (1 + N(0, noise)).

The paper's data (a 131M-history scan of a head phantom, Sec. 3.1; Catphan 404
and CIRS 715HN scans, Sec. 3.2 and 4.3) are not available; these synthetic
workloads stand in for them with the shapes the paper gives (Sec. 2: about 1e9
histories, a few hundred non-zeros per row of a 1-2 million voxel grid).

Geometry conventions (shared by the oracle and the CUDA path as *input*
conventions): the grid is centred at the origin with x fastest; the gantry angle
phi rotates about z; the beam direction is d = (cos phi, sin phi, 0), the
lateral axis e_t = (-sin phi, cos phi, 0) and the vertical axis e_v = (0, 0, 1).
The two measurement planes sit at depth u0 = -R and u2 = +R with
R = min(nx*hx, ny*hy)/2. A record holds t0, v0, st0, sv0 (position in mm and
slope dt/du, dv/du at u0), the same four at u2, the WEPL in mm, and cos/sin phi.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

RECORD_FIELDS = ("t0", "v0", "st0", "sv0", "t2", "v2", "st2", "sv2", "wepl", "cphi", "sphi")
RSP_AIR = 0.001
RSP_WATER = 1.0


@dataclasses.dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float

    @property
    def m(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def radius(self) -> float:
        """Half distance between the measurement planes (inscribed radius)."""
        return min(self.nx * self.hx, self.ny * self.hy) / 2.0

    @property
    def box_min(self) -> np.ndarray:
        return -0.5 * np.array([self.nx * self.hx, self.ny * self.hy, self.nz * self.hz])

    @property
    def box_max(self) -> np.ndarray:
        return -self.box_min

    def voxel_centres(self) -> np.ndarray:
        """(M, 3) voxel centres in mm, x fastest."""
        ix = (np.arange(self.nx) + 0.5) * self.hx + self.box_min[0]
        iy = (np.arange(self.ny) + 0.5) * self.hy + self.box_min[1]
        iz = (np.arange(self.nz) + 0.5) * self.hz + self.box_min[2]
        zz, yy, xx = np.meshgrid(iz, iy, ix, indexing="ij")
        return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


@dataclasses.dataclass(frozen=True)
class Quadric:
    """Axis-aligned ellipsoid (``kind='ellipsoid'``) or infinite z-cylinder
    (``kind='cylz'``, semi-axes (a, b, _)) adding ``delta`` to the RSP inside."""

    kind: str
    centre: Tuple[float, float, float]
    axes: Tuple[float, float, float]
    delta: float


@dataclasses.dataclass(frozen=True)
class Phantom:
    base: float
    parts: Tuple[Quadric, ...]

    def rsp_at(self, pts: np.ndarray) -> np.ndarray:
        out = np.full(pts.shape[0], self.base, dtype=np.float64)
        for q in self.parts:
            out += q.delta * _inside(q, pts)
        return out


def _inside(q: Quadric, pts: np.ndarray) -> np.ndarray:
    c = np.asarray(q.centre)
    a = np.asarray(q.axes, dtype=np.float64)
    r = (pts - c) / a
    if q.kind == "ellipsoid":
        s = (r * r).sum(axis=1)
    elif q.kind == "cylz":
        s = (r[:, :2] ** 2).sum(axis=1)
    else:
        raise ValueError(q.kind)
    return (s < 1.0).astype(np.float64)


def water_cylinder(radius: float = 25.0) -> Phantom:
    """Water cylinder (RSP 1.0) of the given radius, axis z, in air."""
    return Phantom(RSP_AIR, (Quadric("cylz", (0.0, 0.0, 0.0), (radius, radius, 1.0), RSP_WATER - RSP_AIR),))


def head_phantom(seed: int = 0, jitter: float = 0.0) -> Phantom:
    """Ellipsoidal head: 6 mm bone shell (1.6) around tissue (1.04), two
    sinus-like air ellipsoids and two bone inserts. ``jitter`` scales the
    outer semi-axes and the insert positions by up to +-jitter (seeded)."""
    rng = np.random.Generator(np.random.Philox(seed + 0x5EED))
    j = lambda: 1.0 + jitter * (2.0 * rng.random() - 1.0)  # noqa: E731
    A, B, C = 90.0 * j(), 75.0 * j(), 38.0 * j()
    C = min(C, 38.0)
    shell = 6.0
    bone, tissue = 1.6, 1.04
    parts: List[Quadric] = [
        Quadric("ellipsoid", (0.0, 0.0, 0.0), (A, B, C), bone - RSP_AIR),
        Quadric("ellipsoid", (0.0, 0.0, 0.0), (A - shell, B - shell, C - shell), tissue - bone),
    ]
    # Inserts: positions are fractions of the inner semi-axes, jittered.
    Ai, Bi, Ci = A - shell, B - shell, C - shell
    specs = [
        ((+0.45, +0.40, +0.15), (14.0, 10.0, 9.0), RSP_AIR - tissue),
        ((-0.45, +0.40, +0.15), (14.0, 10.0, 9.0), RSP_AIR - tissue),
        ((+0.35, -0.45, -0.20), (9.0, 9.0, 8.0), bone - tissue),
        ((-0.30, -0.40, -0.10), (7.0, 12.0, 7.0), bone - tissue),
    ]
    for (fx, fy, fz), ax, d in specs:
        cx = fx * Ai * j()
        cy = fy * Bi * j()
        cz = fz * Ci * j()
        parts.append(Quadric("ellipsoid", (cx, cy, cz), ax, d))
    return Phantom(RSP_AIR, tuple(parts))


# Inserts with the "true" RSPs of Table 2 (Sec. 4.2); the layout (a ring of
# 12 mm cylinders at 50 mm from the axis of a 150 mm water-equivalent
# cylinder) is a chosen one: the paper shows the phantom (Fig. 3) only as an image.
CATPHAN_INSERTS = (("Teflon", 1.790), ("PMP", 0.883), ("LDPE", 0.979), ("Polystyrene", 1.024),
                   ("Delrin", 1.359), ("Air 1", 0.00113), ("Air 2", 0.00113))
CATPHAN_BODY = 1.0
CATPHAN_RADIUS = 75.0
INSERT_RADIUS = 6.0
INSERT_RING = 50.0


def insert_centres():
    n = len(CATPHAN_INSERTS)
    return [(INSERT_RING * math.cos(2 * math.pi * k / n), INSERT_RING * math.sin(2 * math.pi * k / n))
            for k in range(n)]


def catphan_phantom() -> Phantom:
    """Cylinder of RSP 1.0 (r = 75 mm, axis z) with seven r = 6 mm cylindrical
    inserts at the true RSPs of Table 2, in air."""
    parts = [Quadric("cylz", (0.0, 0.0, 0.0), (CATPHAN_RADIUS, CATPHAN_RADIUS, 1.0), CATPHAN_BODY - RSP_AIR)]
    for (name, rsp), (cx, cy) in zip(CATPHAN_INSERTS, insert_centres()):
        parts.append(Quadric("cylz", (cx, cy, 0.0), (INSERT_RADIUS, INSERT_RADIUS, 1.0), rsp - CATPHAN_BODY))
    return Phantom(RSP_AIR, tuple(parts))


def roi_stats(x: np.ndarray, grid: Grid, margin_mm: float = 2.0, z_margin_mm: float = 5.0):
    """Table 2 style ROI analysis: for each insert, the voxels whose centres lie
    in a cylinder of radius (6 mm - margin) around the insert axis and more than
    z_margin from the grid's top and bottom (away from partial volume). Returns
    rows (name, true, mean, std, %error)."""
    c = grid.voxel_centres()
    zmax = 0.5 * grid.nz * grid.hz - z_margin_mm
    rows = []
    for (name, rsp), (cx, cy) in zip(CATPHAN_INSERTS, insert_centres()):
        m = ((c[:, 0] - cx) ** 2 + (c[:, 1] - cy) ** 2 <= (INSERT_RADIUS - margin_mm) ** 2) & (np.abs(c[:, 2]) <= zmax)
        v = x[m]
        mean = float(v.mean())
        err = 100.0 * (mean - rsp) / rsp if rsp > 0.01 else None
        rows.append({"material": name, "true": rsp, "mean": mean, "std": float(v.std()), "pct_error": err,
                     "voxels": int(m.sum())})
    return rows


def voxelize(ph: Phantom, grid: Grid, ss: int = 3) -> np.ndarray:
    """Voxel-average RSP by ss^3 supersampling; float64 array of length M."""
    out = np.zeros(grid.m, dtype=np.float64)
    c = grid.voxel_centres()
    h = np.array([grid.hx, grid.hy, grid.hz])
    offs = (np.arange(ss) + 0.5) / ss - 0.5
    for ox in offs:
        for oy in offs:
            for oz in offs:
                out += ph.rsp_at(c + h * np.array([ox, oy, oz]))
    return out / ss ** 3


def interior_mask(x_true: np.ndarray, grid: Grid, thr: float = 0.5) -> np.ndarray:
    """Voxels with x_true >= thr whose 3x3x3 neighbourhood is one material
    (more than one voxel from any boundary): the ROI of the mean-error metric."""
    v = x_true.reshape(grid.nz, grid.ny, grid.nx)
    ok = v >= thr
    same = np.ones_like(ok)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                sh = np.roll(np.roll(np.roll(v, dz, 0), dy, 1), dx, 2)
                same &= np.abs(sh - v) < 1e-9
    edge = np.zeros_like(ok)
    edge[[0, -1], :, :] = True
    edge[:, [0, -1], :] = True
    edge[:, :, [0, -1]] = True
    return (ok & same & ~edge).ravel()


def mean_rsp_error(x: np.ndarray, x_true: np.ndarray, grid: Grid) -> float:
    """Mean relative RSP error over the interior ROI (partial-volume free)."""
    m = interior_mask(x_true, grid)
    return float(np.mean(np.abs(x[m] - x_true[m]) / x_true[m]))


def _chord_quadric(q: Quadric, p0: np.ndarray, dv: np.ndarray, ta: np.ndarray, tb: np.ndarray) -> np.ndarray:
    """Length of {p0 + tau*dv : tau in [ta, tb]} inside the quadric (vectorised)."""
    c = np.asarray(q.centre)
    a = np.asarray(q.axes, dtype=np.float64)
    o = (p0 - c) / a
    d = dv / a
    if q.kind == "cylz":
        o = o[:, :2]
        d = d[:, :2]
    A = (d * d).sum(axis=1)
    Bq = 2.0 * (o * d).sum(axis=1)
    Cq = (o * o).sum(axis=1) - 1.0
    disc = Bq * Bq - 4.0 * A * Cq
    ok = (disc > 0) & (A > 0)
    sq = np.sqrt(np.where(ok, disc, 0.0))
    Asafe = np.where(A > 0, A, 1.0)
    t1 = (-Bq - sq) / (2.0 * Asafe)
    t2 = (-Bq + sq) / (2.0 * Asafe)
    lo = np.maximum(t1, ta)
    hi = np.minimum(t2, tb)
    L = np.linalg.norm(dv, axis=1)
    return np.where(ok & (hi > lo), (hi - lo) * L, 0.0)


def _box_clip(grid: Grid, p0: np.ndarray, dv: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Parameter interval of the infinite line p0 + tau*dv inside the grid box."""
    lo = np.full(p0.shape[0], -np.inf)
    hi = np.full(p0.shape[0], np.inf)
    bmin, bmax = grid.box_min, grid.box_max
    for a in range(3):
        d = dv[:, a]
        nz = d != 0
        dsafe = np.where(nz, d, 1.0)
        t1 = (bmin[a] - p0[:, a]) / dsafe
        t2 = (bmax[a] - p0[:, a]) / dsafe
        tmin = np.where(nz, np.minimum(t1, t2), np.where((p0[:, a] >= bmin[a]) & (p0[:, a] <= bmax[a]), -np.inf, np.inf))
        tmax = np.where(nz, np.maximum(t1, t2), np.where((p0[:, a] >= bmin[a]) & (p0[:, a] <= bmax[a]), np.inf, -np.inf))
        lo = np.maximum(lo, tmin)
        hi = np.minimum(hi, tmax)
    return lo, hi


def straight_wepl(ph: Phantom, grid: Grid, rec: Dict[str, np.ndarray]) -> np.ndarray:
    """RSP line integral along the straight line through the entry point (at
    u0) and the exit point (at u2), over the part of that line in the grid box."""
    R = grid.radius
    c = rec["cphi"].astype(np.float64)
    s = rec["sphi"].astype(np.float64)

    def point(u, t, v):
        return np.stack([u * c - t * s, u * s + t * c, v], axis=1)

    p0 = point(-R, rec["t0"].astype(np.float64), rec["v0"].astype(np.float64))
    p2 = point(+R, rec["t2"].astype(np.float64), rec["v2"].astype(np.float64))
    dv = p2 - p0
    ta, tb = _box_clip(grid, p0, dv)
    L = np.linalg.norm(dv, axis=1)
    out = ph.base * np.maximum(tb - ta, 0.0) * L
    for q in ph.parts:
        out += q.delta * _chord_quadric(q, p0, dv, ta, tb)
    return out


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic workload: grid, phantom, history count and recipe."""

    name: str
    grid: Grid
    n: int
    seed: int
    n_angles: int  # 0 = continuous angles
    t_range: float
    v_range: float
    n_blocks: int
    n_sweeps: int
    phantom_kind: str = "water"
    jitter: float = 0.0

    def phantom(self) -> Phantom:
        if self.phantom_kind == "water":
            return water_cylinder(25.0)
        if self.phantom_kind == "head":
            return head_phantom(self.seed, self.jitter)
        if self.phantom_kind == "catphan":
            return catphan_phantom()
        raise ValueError(self.phantom_kind)


def tiny_workload(n: int = 100_000, seed: int = 1) -> Workload:
    """32^3 grid of 2 mm voxels, water cylinder r = 25 mm; 10 blocks, 10 sweeps."""
    return Workload("water32_100k", Grid(32, 32, 32, 2.0, 2.0, 2.0), n, seed, 0, 30.0, 30.0, 10, 10, "water")


def head_workload(n: int = 50_000_000, seed: int = 2) -> Workload:
    """160x160x64 grid of 1.25 mm voxels (1.64M voxels), ellipsoid head,
    90 projection angles; 10 blocks, 10 sweeps."""
    g = Grid(160, 160, 64, 1.25, 1.25, 1.25)
    return Workload(f"head160_{n}", g, n, seed, 90, g.radius, 40.0, 10, 10, "head")


def head200_workload(n: int = 1_000_000_000, seed: int = 5, n_blocks: int = 50) -> Workload:
    """200x200x48 grid of 1 x 1 x 2 mm voxels (1.92M voxels), a seeded random
    head (outer semi-axes and inserts jittered by +-15 %), 90 projection
    angles, vertical entry positions within +-46 mm; 1e9 histories and 50
    blocks by default."""
    g = Grid(200, 200, 48, 1.0, 1.0, 2.0)
    return Workload(f"head200x200x48_{n}", g, n, seed, 90, g.radius, min(46.0, 0.5 * g.nz * g.hz - 2.0), n_blocks,
                    10, "head", 0.15)


def batch_workloads(n_recon: int = 32, seed: int = 4, n_min: int = 2_000_000, n_max: int = 40_000_000,
                    n_blocks: int = 10):
    """Independent reconstructions of uneven size: grids from 64x64x32 to
    160x160x64 voxels over a 200 mm field (nx log-uniform, nz = 0.4 nx clamped
    to [32, 64]) and 2M-40M histories each (log-uniform), seeded; random head
    phantoms (+-10 % jitter), 90 angles."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for r in range(n_recon):
        nx = int(round(math.exp(rng.uniform(math.log(64), math.log(160))) / 8.0)) * 8
        nx = min(160, max(64, nx))
        nz = min(64, max(32, int(round(0.4 * nx / 2.0)) * 2))
        h = 200.0 / nx
        n = int(math.exp(rng.uniform(math.log(n_min), math.log(n_max))))
        g = Grid(nx, nx, nz, h, h, h)
        out.append(Workload(f"batch{r}_{nx}x{nx}x{nz}_{n}", g, n, seed * 1000 + r, 90, g.radius,
                            min(40.0, 0.5 * nz * h - 2.0), n_blocks, 10, "head", 0.1))
    return out


def slab_sigma(length_mm: float) -> Tuple[float, float]:
    """Generator recipe for the exit-state spread: slope sigma 14.7 mrad for
    a 64 mm slab scaled by sqrt(length/64 mm); returned with the length."""
    return 0.0147 * math.sqrt(length_mm / 64.0), length_mm


def make_histories(wl: Workload, n: int | None = None, seed_offset: int = 0, noise: float = 0.01,
                   slope_sigma: float = 0.003) -> Dict[str, np.ndarray]:
    """Generate ``n`` (default ``wl.n``) float32 SoA records for ``wl``.

    Entry: t0 ~ U(+-t_range), v0 ~ U(+-v_range), slopes ~ N(0, slope_sigma).
    Exit: straight continuation plus a correlated Gaussian (t, slope) kick with
    covariance sigma^2 [[L^2/3, L/2], [L/2, 1]] (L = 2R). phi is uniform on
    [0, 2pi) (``n_angles == 0``) or one of ``n_angles`` equispaced angles, in
    random order so every contiguous block spans all angles.
    """
    n = wl.n if n is None else n
    g = wl.grid
    R = g.radius
    rng = np.random.Generator(np.random.Philox(wl.seed * 1_000_003 + seed_offset))
    if wl.n_angles == 0:
        phi = rng.random(n) * (2.0 * math.pi)
    else:
        phi = rng.integers(0, wl.n_angles, n) * (2.0 * math.pi / wl.n_angles)
    t0 = (2.0 * rng.random(n) - 1.0) * wl.t_range
    v0 = (2.0 * rng.random(n) - 1.0) * wl.v_range
    st0 = rng.standard_normal(n) * slope_sigma
    sv0 = rng.standard_normal(n) * slope_sigma
    sig, L = slab_sigma(2.0 * R)
    out = {"t0": t0, "v0": v0, "st0": st0, "sv0": sv0}
    for lat, pos, slope in (("t", t0, st0), ("v", v0, sv0)):
        z1 = rng.standard_normal(n)
        z2 = rng.standard_normal(n)
        ds = sig * z1
        dt = sig * L * (0.5 * z1 + z2 / (2.0 * math.sqrt(3.0)))
        out[lat + "2"] = pos + L * slope + dt
        out["s" + lat + "2"] = slope + ds
    out["cphi"] = np.cos(phi)
    out["sphi"] = np.sin(phi)
    rec = {k: np.ascontiguousarray(v, dtype=np.float32) for k, v in out.items()}
    w = straight_wepl(wl.phantom(), g, rec)
    w = w * (1.0 + noise * rng.standard_normal(n))
    rec["wepl"] = np.maximum(w, 0.0).astype(np.float32)
    return {k: rec[k] for k in RECORD_FIELDS}


def straight_records(grid: Grid, t: Sequence[float], v: Sequence[float], s_t: Sequence[float],
                     s_v: Sequence[float], phi: Sequence[float]) -> Dict[str, np.ndarray]:
    """Consistent straight-line records (exit = entry + 2R * slope, equal
    slopes); WEPL 0. Used by the straight-line-limit pins."""
    R = grid.radius
    t = np.asarray(t, np.float64)
    v = np.asarray(v, np.float64)
    s_t = np.asarray(s_t, np.float64)
    s_v = np.asarray(s_v, np.float64)
    phi = np.asarray(phi, np.float64)
    rec = {
        "t0": t, "v0": v, "st0": s_t, "sv0": s_v,
        "t2": t + 2 * R * s_t, "v2": v + 2 * R * s_v, "st2": s_t, "sv2": s_v,
        "wepl": np.zeros_like(t), "cphi": np.cos(phi), "sphi": np.sin(phi),
    }
    return {k: np.ascontiguousarray(rec[k], dtype=np.float32) for k in RECORD_FIELDS}


def concat(recs: Sequence[Dict[str, np.ndarray]]) -> Dict[str, np.ndarray]:
    return {k: np.concatenate([r[k] for r in recs]) for k in RECORD_FIELDS}


def subset(rec: Dict[str, np.ndarray], idx) -> Dict[str, np.ndarray]:
    return {k: np.ascontiguousarray(rec[k][idx]) for k in RECORD_FIELDS}


# ---------------------------------------------------------------------------
# Device-side generator (same recipe, torch RNG on the GPU) for large N.
# ---------------------------------------------------------------------------

def _chord_quadric_t(torch, q: Quadric, p0, dv, ta, tb):
    c = torch.tensor(q.centre, dtype=p0.dtype, device=p0.device)
    a = torch.tensor(q.axes, dtype=p0.dtype, device=p0.device)
    o = (p0 - c) / a
    d = dv / a
    if q.kind == "cylz":
        o = o[:, :2]
        d = d[:, :2]
    A = (d * d).sum(dim=1)
    Bq = 2.0 * (o * d).sum(dim=1)
    Cq = (o * o).sum(dim=1) - 1.0
    disc = Bq * Bq - 4.0 * A * Cq
    ok = (disc > 0) & (A > 0)
    sq = torch.sqrt(torch.where(ok, disc, torch.zeros_like(disc)))
    Asafe = torch.where(A > 0, A, torch.ones_like(A))
    t1 = (-Bq - sq) / (2.0 * Asafe)
    t2 = (-Bq + sq) / (2.0 * Asafe)
    lo = torch.maximum(t1, ta)
    hi = torch.minimum(t2, tb)
    L = torch.linalg.norm(dv, dim=1)
    return torch.where(ok & (hi > lo), (hi - lo) * L, torch.zeros_like(L))


def _box_clip_t(torch, grid: Grid, p0, dv):
    n = p0.shape[0]
    inf = torch.full((n,), float("inf"), dtype=p0.dtype, device=p0.device)
    lo, hi = -inf, inf.clone()
    bmin, bmax = grid.box_min, grid.box_max
    for a in range(3):
        d = dv[:, a]
        nz = d != 0
        dsafe = torch.where(nz, d, torch.ones_like(d))
        t1 = (float(bmin[a]) - p0[:, a]) / dsafe
        t2 = (float(bmax[a]) - p0[:, a]) / dsafe
        inside = (p0[:, a] >= float(bmin[a])) & (p0[:, a] <= float(bmax[a]))
        tmin = torch.where(nz, torch.minimum(t1, t2), torch.where(inside, -inf, inf))
        tmax = torch.where(nz, torch.maximum(t1, t2), torch.where(inside, inf, -inf))
        lo = torch.maximum(lo, tmin)
        hi = torch.minimum(hi, tmax)
    return lo, hi


def make_histories_device(wl: Workload, n: int | None = None, device: str = "cuda", seed_offset: int = 0,
                          noise: float = 0.01, slope_sigma: float = 0.003, chunk: int = 8_000_000):
    """Same recipe as :func:`make_histories`, drawn with torch's generator on
    ``device`` (a different random stream). Returns float32 tensors."""
    import torch

    n = wl.n if n is None else n
    g = wl.grid
    R = g.radius
    gen = torch.Generator(device=device)
    gen.manual_seed(wl.seed * 1_000_003 + seed_offset)
    ph = wl.phantom()
    sig, L = slab_sigma(2.0 * R)
    out = {f: torch.empty(n, dtype=torch.float32, device=device) for f in RECORD_FIELDS}
    f64 = torch.float64
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        rnd = lambda: torch.rand(m, generator=gen, device=device, dtype=f64)  # noqa: E731
        nrm = lambda: torch.randn(m, generator=gen, device=device, dtype=f64)  # noqa: E731
        if wl.n_angles == 0:
            phi = rnd() * (2.0 * math.pi)
        else:
            phi = torch.randint(0, wl.n_angles, (m,), generator=gen, device=device).to(f64) * (2.0 * math.pi / wl.n_angles)
        t0 = (2.0 * rnd() - 1.0) * wl.t_range
        v0 = (2.0 * rnd() - 1.0) * wl.v_range
        st0 = nrm() * slope_sigma
        sv0 = nrm() * slope_sigma
        part = {"t0": t0, "v0": v0, "st0": st0, "sv0": sv0}
        for lat, pos, slope in (("t", t0, st0), ("v", v0, sv0)):
            z1 = nrm()
            z2 = nrm()
            part[lat + "2"] = pos + L * slope + sig * L * (0.5 * z1 + z2 / (2.0 * math.sqrt(3.0)))
            part["s" + lat + "2"] = slope + sig * z1
        part["cphi"] = torch.cos(phi)
        part["sphi"] = torch.sin(phi)
        r32 = {k: v.to(torch.float32) for k, v in part.items()}
        c = r32["cphi"].to(f64)
        sn = r32["sphi"].to(f64)
        p0 = torch.stack([-R * c - r32["t0"].to(f64) * sn, -R * sn + r32["t0"].to(f64) * c, r32["v0"].to(f64)], 1)
        p2 = torch.stack([R * c - r32["t2"].to(f64) * sn, R * sn + r32["t2"].to(f64) * c, r32["v2"].to(f64)], 1)
        dv = p2 - p0
        ta, tb = _box_clip_t(torch, g, p0, dv)
        w = ph.base * torch.clamp(tb - ta, min=0.0) * torch.linalg.norm(dv, dim=1)
        for q in ph.parts:
            w = w + q.delta * _chord_quadric_t(torch, q, p0, dv, ta, tb)
        w = w * (1.0 + noise * nrm())
        r32["wepl"] = torch.clamp(w, min=0.0).to(torch.float32)
        for k in RECORD_FIELDS:
            out[k][s:s + m] = r32[k]
    return out
