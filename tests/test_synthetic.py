"""Input-generator checks: the insert phantom and its Table 2 style ROI
analysis, straight-line WEPL against a brute-force line integral, and the
device generator against the host recipe."""
import math

import numpy as np

from paper_1707_05014_gb300 import synthetic as S


def test_roi_stats_on_the_true_image_are_exact():
    g = S.Grid(160, 160, 32, 1.25, 1.25, 1.25)
    x = S.voxelize(S.catphan_phantom(), g, ss=2)
    rows = S.roi_stats(x, g)
    assert [r["material"] for r in rows] == [m for m, _ in S.CATPHAN_INSERTS]
    for r in rows:
        assert r["voxels"] > 100
        assert abs(r["mean"] - r["true"]) < 1e-12 and r["std"] < 1e-12
        if r["pct_error"] is not None:
            assert abs(r["pct_error"]) < 1e-9


def test_straight_wepl_matches_brute_force_integral():
    wl = S.head_workload(50, seed=3)
    g = wl.grid
    rec = S.make_histories(wl, noise=0.0)
    ph = wl.phantom()
    R = g.radius
    for i in range(10):
        c, s = float(rec["cphi"][i]), float(rec["sphi"][i])
        p0 = np.array([-R * c - float(rec["t0"][i]) * s, -R * s + float(rec["t0"][i]) * c, float(rec["v0"][i])])
        p2 = np.array([R * c - float(rec["t2"][i]) * s, R * s + float(rec["t2"][i]) * c, float(rec["v2"][i])])
        d = p2 - p0
        # sample the whole line through the box with a fine step
        ts = np.linspace(-2.0, 3.0, 400_001)
        pts = p0[None, :] + ts[:, None] * d[None, :]
        inside = np.all((pts >= g.box_min) & (pts <= g.box_max), axis=1)
        dl = (ts[1] - ts[0]) * np.linalg.norm(d)
        ref = float(ph.rsp_at(pts[inside]).sum() * dl)
        assert abs(float(rec["wepl"][i]) - ref) <= 2e-3 * max(ref, 1.0)
