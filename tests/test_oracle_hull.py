"""Pins for the oracle's object-hull path.

The MLP literature the paper cites (Sec. 2: Williams 2004, Schulte 2008)
estimates the path inside the object only; outside it the proton flies
straight. With a hull, each proton's MLP runs between the first node of its
entry ray and the last node of its exit ray that lie in hull voxels, using the
table of a water layer of that thickness; without one (or for a proton that
misses the hull) it runs between the measurement planes. Checks here use
closed-form moments and Gaussian conditioning (independent of the oracle's
quadrature and matrix route), exact invariances, a numpy re-derivation of the
hull ranges, and reductions to the hull-free path.
"""
import math

import numpy as np
import pytest
from test_oracle_mlp import E0, X0, _closed_moment

from paper_1707_05014_gb300 import synthetic as S

G_TINY = S.Grid(32, 32, 32, 2.0, 2.0, 2.0)
G_HEAD = S.Grid(160, 160, 64, 1.25, 1.25, 1.25)


def _kalman_layer(du, n, W):
    """Gaussian-conditioning MLP coefficients of nodes m = 0..n, spaced du mm,
    in a water layer W cm thick, from closed-form moments."""
    out = np.zeros((n + 1, 4))
    out[0] = (1, 0, 0, 0)
    out[n] = (0, 0, 1, 0)
    hl = lambda L: E0 * E0 * (1 + 0.038 * math.log(L / X0)) ** 2 / X0  # noqa: E731
    for m in range(1, n):
        w1 = m * du / 10.0
        S1 = hl(w1) * np.array([[_closed_moment(0, w1, w1, 2), _closed_moment(0, w1, w1, 1)],
                                [_closed_moment(0, w1, w1, 1), _closed_moment(0, w1, w1, 0)]])
        S2 = hl(W - w1) * np.array([[_closed_moment(w1, W, W, 2), _closed_moment(w1, W, W, 1)],
                                    [_closed_moment(w1, W, W, 1), _closed_moment(w1, W, W, 0)]])
        R0 = np.array([[1.0, w1], [0.0, 1.0]])
        R1 = np.array([[1.0, W - w1], [0.0, 1.0]])
        C = R1 @ S1 @ R1.T + S2
        G = S1 @ R1.T @ np.linalg.inv(C)
        A0 = (np.eye(2) - G @ R1) @ R0
        out[m] = (A0[0, 0], 10 * A0[0, 1], G[0, 0], 10 * G[0, 1])
    return out


def test_layer_table_of_the_slab_is_the_plane_table(oracle):
    for g in (G_TINY, G_HEAD):
        _, _, K, _ = oracle.geom_info(g)
        assert np.array_equal(oracle.mlp_table_n(g, K), oracle.mlp_table(g))


@pytest.mark.parametrize("frac", [0.02, 0.3, 0.71, 0.97])
def test_layer_tables_equal_conditioning_form_and_invariances(oracle, frac):
    g = G_HEAD
    _, du, K, _ = oracle.geom_info(g)
    n = max(1, int(frac * K))
    tab = oracle.mlp_table_n(g, n)
    ref = _kalman_layer(du, n, n * du / 10.0)
    L = n * du
    assert np.abs((tab - ref) / np.array([1.0, L, 1.0, L])).max() < 1e-12
    # translation and straight-line invariance over the layer
    m = np.arange(n + 1) * du
    assert np.abs(tab[:, 0] + tab[:, 2] - 1.0).max() < 1e-12
    assert np.abs(tab[:, 1] + tab[:, 2] * L + tab[:, 3] - m).max() < 1e-12 * L
    assert tuple(tab[0]) == (1.0, 0.0, 0.0, 0.0) and tuple(tab[n]) == (0.0, 0.0, 1.0, 0.0)


def test_layer_depth_reversal_with_constant_scattering(oracle):
    g = G_HEAD
    _, du, K, _ = oracle.geom_info(g)
    for n in (7, 150):
        tab = oracle.mlp_table_n(g, n, flags=oracle.F_CONST_SCATTER)
        rev = tab[::-1]
        assert np.abs(tab[:, 0] - rev[:, 2]).max() < 1e-12
        assert np.abs(tab[:, 1] + rev[:, 3]).max() < 1e-12 * n * du


def _hull_mask(g, ph, thr=0.5):
    return (S.voxelize(ph, g, ss=1) > thr).astype(np.uint8)


def _ranges_numpy(g, rec, hull, du, K):
    """FP64 hull ranges re-derived with numpy: first entry-ray node k in
    [0, K] in a hull voxel, last exit-ray node in one; (0, K) otherwise."""
    R = g.radius
    n = len(rec["t0"])
    k = np.arange(K + 1, dtype=np.float64)
    u = -R + k * du
    out = np.zeros((n, 2), dtype=np.int64)
    h3 = hull.reshape(g.nz, g.ny, g.nx)
    for i in range(n):
        c, s = float(rec["cphi"][i]), float(rec["sphi"][i])
        hits = []
        for (t0, s0, v0, sv, off) in ((rec["t0"][i], rec["st0"][i], rec["v0"][i], rec["sv0"][i], 0),
                                      (rec["t2"][i], rec["st2"][i], rec["v2"][i], rec["sv2"][i], K)):
            t = float(t0) + float(s0) * ((k - off) * du)
            v = float(v0) + float(sv) * ((k - off) * du)
            q = np.stack([(u * c - t * s) / g.hx + g.nx / 2, (u * s + t * c) / g.hy + g.ny / 2, v / g.hz + g.nz / 2])
            ix, iy, iz = (np.floor(np.round(q * 2.0**20) / 2.0**20).astype(np.int64))
            ok = (ix >= 0) & (ix < g.nx) & (iy >= 0) & (iy < g.ny) & (iz >= 0) & (iz < g.nz)
            inside = np.zeros(K + 1, bool)
            inside[ok] = h3[iz[ok], iy[ok], ix[ok]] != 0
            hits.append(np.flatnonzero(inside))
        if len(hits[0]) and len(hits[1]) and hits[1][-1] > hits[0][0]:
            out[i] = (hits[0][0], hits[1][-1])
        else:
            out[i] = (0, K)
    return out


def test_hull_ranges_match_numpy(oracle):
    wl = S.tiny_workload(400, seed=11)
    g = wl.grid
    rec = S.make_histories(wl)
    hull = _hull_mask(g, wl.phantom())
    _, du, K, _ = oracle.geom_info(g)
    got = oracle.hull_ranges(g, rec, hull, mode=oracle.MODE_FP64)
    ref = _ranges_numpy(g, rec, hull, du, K)
    assert np.array_equal(got, ref)
    # the cylinder is thinner than the slab: most protons that hit it enter
    # after the first plane and leave before the second
    hit = (got[:, 0] > 0) & (got[:, 1] < K)
    assert hit.mean() > 0.5
    # FP32 and FP64 node orders agree on the ranges up to boundary ties
    r32 = oracle.hull_ranges(g, rec, hull, mode=oracle.MODE_FP32)
    assert (r32 != got).any(axis=1).mean() < 0.01


def test_full_range_and_missing_protons_keep_the_plane_path(oracle):
    wl = S.tiny_workload(300, seed=12)
    g = wl.grid
    rec = S.make_histories(wl)
    _, _, K, _ = oracle.geom_info(g)
    # hull = the whole grid: protons whose rays are inside the grid at both
    # planes have range (0, K) and keep their rows exactly
    full = np.ones(g.nx * g.ny * g.nz, np.uint8)
    rng = oracle.hull_ranges(g, rec, full)
    keep = np.flatnonzero((rng[:, 0] == 0) & (rng[:, 1] == K))
    assert len(keep) > 50
    sub = S.subset(rec, keep)
    a = oracle.rows(g, sub)
    b = oracle.rows(g, sub, hull=full)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    # an empty hull: every proton misses it and keeps its rows
    empty = np.zeros_like(full)
    assert np.array_equal(oracle.hull_ranges(g, rec, empty), np.tile([0, K], (300, 1)))
    c = oracle.rows(g, rec, hull=empty)
    d = oracle.rows(g, rec)
    assert np.array_equal(c[1], d[1]) and np.array_equal(c[2], d[2])


def test_straight_records_stay_straight_inside_a_hull(oracle):
    g = G_HEAD
    R, du, K, _ = oracle.geom_info(g)
    hull = _hull_mask(g, S.head_phantom())
    rec = S.straight_records(g, [10.0, -33.0], [5.0, -12.0], [0.02, -0.01], [0.0, 0.015], [0.3, 2.0])
    rng = oracle.hull_ranges(g, rec, hull, mode=oracle.MODE_FP64)
    assert np.all(rng[:, 0] > 0) and np.all(rng[:, 1] < K)
    q = oracle.nodes(g, rec, mode=oracle.MODE_FP64, hull=hull).astype(np.float64) / 2.0**20
    for i in range(2):
        c, s = float(rec["cphi"][i]), float(rec["sphi"][i])
        u = -R + np.arange(K + 1) * du
        t = float(rec["t0"][i]) + float(rec["st0"][i]) * (u + R)
        v = float(rec["v0"][i]) + float(rec["sv0"][i]) * (u + R)
        ref = np.stack([(u * c - t * s) / g.hx + g.nx / 2, (u * s + t * c) / g.hy + g.ny / 2, v / g.hz + g.nz / 2], 1)
        assert np.abs(q[i] - ref).max() < 5e-6


def test_hull_changes_only_the_estimate_inside_the_object(oracle):
    # With a hull, nodes up to the entry and from the exit lie on the measured
    # rays; between them the path differs from the plane-to-plane MLP.
    wl = S.head_workload(200, seed=13)
    g = wl.grid
    rec = S.make_histories(wl)
    R, du, K, _ = oracle.geom_info(g)
    hull = _hull_mask(g, wl.phantom())
    rng = oracle.hull_ranges(g, rec, hull, mode=oracle.MODE_FP64)
    qh = oracle.nodes(g, rec, mode=oracle.MODE_FP64, hull=hull).astype(np.float64) / 2.0**20
    qp = oracle.nodes(g, rec, mode=oracle.MODE_FP64).astype(np.float64) / 2.0**20
    moved = 0
    for i in range(200):
        a, b = rng[i]
        c, s = float(rec["cphi"][i]), float(rec["sphi"][i])
        u = -R + np.arange(K + 1) * du
        for lo, hi, t0, s0, off in ((0, a + 1, "t0", "st0", 0), (b, K + 1, "t2", "st2", K)):
            t = float(rec[t0][i]) + float(rec[s0][i]) * ((np.arange(K + 1) - off) * du)
            x = (u * c - t * s) / g.hx + g.nx / 2
            assert np.abs(qh[i, lo:hi, 0] - x[lo:hi]).max() < 5e-6
        if b - a < K:
            moved += np.abs(qh[i, a + 1:b] - qp[i, a + 1:b]).max() > 1e-3
    assert moved > 100


def test_carved_hull_contains_the_object(oracle):
    wl = S.tiny_workload(20_000, seed=14)
    g = wl.grid
    rec = S.make_histories(wl, noise=0.0)
    xt = S.voxelize(wl.phantom(), g)
    hull = oracle.carve_hull(g, rec, wepl_max=1.0, dilate=1)
    assert np.all(hull[xt >= 0.5] == 1)
    # air far from the cylinder (r > 35 mm) is carved away, in the slices the
    # histories cover (|v| <= 30 mm on a 64 mm tall grid)
    c = (np.arange(g.nx) + 0.5) * g.hx - g.nx * g.hx / 2
    z = (np.arange(g.nz) + 0.5) * g.hz - g.nz * g.hz / 2
    r2 = c[None, None, :] ** 2 + c[None, :, None] ** 2
    far = ((r2 > 35.0**2) & (np.abs(z) < 24.0)[:, None, None]).reshape(-1)
    h0 = oracle.carve_hull(g, rec, wepl_max=1.0, dilate=0)
    assert h0[far].mean() < 0.1
    # dilation only grows the hull
    assert np.all(hull[h0 == 1] == 1) and h0.sum() < hull.sum()


def test_hull_drop_consistent_data_converges(oracle):
    wl = S.tiny_workload(4000, seed=15)
    g = wl.grid
    rec = S.make_histories(wl)
    xt = S.voxelize(wl.phantom(), g)
    hull = _hull_mask(g, wl.phantom())
    rec["wepl"] = oracle.project(g, rec, xt, hull=hull).astype(np.float32)
    x, res = oracle.drop(g, rec, 5, 30, lam=1.0, return_resid=True, hull=hull)
    assert np.all(np.diff(res[1:]) < 0)
    assert res[-1] < 2e-3 * res[0]
