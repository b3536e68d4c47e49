"""Input-generator checks: the insert phantom and its Table 2 style ROI
analysis, straight-line WEPL against a brute-force line integral, and the
device generator against the host recipe."""
import math
import os

import numpy as np

from paper_1707_05014_gb300 import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table2_true_rsp():
    """Sec. 4.2, Table 2: the inserts' true RSPs (tests/golden/table2_true_rsp.txt)."""
    out = []
    with open(os.path.join(GOLDEN, "table2_true_rsp.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, rsp = line.rstrip("\n").split("\t")
                out.append((name, float(rsp)))
    return out


def test_insert_phantom_carries_table2_true_rsps():
    # the phantom's materials are the paper's, in the paper's order
    assert list(S.CATPHAN_INSERTS) == _table2_true_rsp()
    # and the voxelised image holds exactly those values at each insert axis
    g = S.Grid(160, 160, 32, 1.25, 1.25, 1.25)
    x = S.voxelize(S.catphan_phantom(), g, ss=1).reshape(g.nz, g.ny, g.nx)
    for (name, rsp), (cx, cy) in zip(_table2_true_rsp(), S.insert_centres()):
        ix = int((cx + 0.5 * g.nx * g.hx) // g.hx)
        iy = int((cy + 0.5 * g.ny * g.hy) // g.hy)
        assert abs(x[g.nz // 2, iy, ix] - rsp) < 1e-12, name


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
