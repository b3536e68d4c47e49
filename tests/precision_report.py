"""Error budget of the FP32 fused path against the FP64 oracle, for the
precision variant of the head workload (160 x 160 x 64 grid of 1.25 mm, 40
blocks, 8 sweeps), on a host-generated subset of its histories:

* MLP nodes (Q20) against FP64 nodes: max and rms in voxels;
* index lists identical to the FP64-node oracle's, and the chord error of
  those that are;
* a_i.x with and without Kahan compensation against an FP64 sum over the same
  rows, and against the full FP64 oracle;
* the image after the 8 sweeps against the FP64 oracle's, and both against
  the phantom.

Test infrastructure (it runs the oracle); needs a GPU. tests/test_gpu_precision.py
asserts the budget on a 200k-history subset; run as a script it prints one JSON
object for a larger subset.

    python tests/precision_report.py [--subset 1000000] [--device 0]
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def report(ns: int = 1_000_000, local: int = 0) -> dict:
    import numpy as np
    import torch

    import oracle as O
    from paper_1707_05014_gb300 import build as B
    from paper_1707_05014_gb300 import pct as P
    from paper_1707_05014_gb300 import synthetic as S

    torch.cuda.set_device(local)
    B.build()
    O.build()
    n_full = 250_000_000
    base = S.head_workload(n_full, seed=3)
    wl = S.Workload(f"head160_precision_{n_full}", base.grid, n_full, 3, 90, base.t_range, base.v_range, 40, 8,
                    "head")
    g = wl.grid
    sub = S.make_histories(wl, n=ns, seed_offset=11)
    x_true = S.voxelize(wl.phantom(), g, ss=2)
    prec = {"subset_histories": ns}
    with P.Context(g, n_blocks=40, device=local) as c:
        c.load(sub)
        k = min(ns, 20_000)
        rp, vox, ln, nodes = (t.cpu().numpy() for t in c.rows(0, k, with_nodes=True))
        n64 = O.nodes(g, sub, 0, k, mode=O.MODE_FP64).astype(np.int64)
        dq = np.abs(nodes.astype(np.int64) - n64) / 2.0**20
        prec["node_error_voxels"] = {"max": float(dq.max()), "rms": float(np.sqrt((dq**2).mean()))}
        orp, ovox, oln = O.rows(g, sub, 0, k, mode=O.MODE_FP64)
        same, d = 0, []
        for i in range(k):
            a, b = vox[rp[i]:rp[i + 1]], ovox[orp[i]:orp[i + 1]]
            if len(a) == len(b) and np.array_equal(a, b):
                same += 1
                d.append(np.abs(ln[rp[i]:rp[i + 1]] - oln[orp[i]:orp[i + 1]]) / np.maximum(oln[orp[i]:orp[i + 1]], g.hx))
        d = np.concatenate(d)
        prec["index_lists_identical_to_fp64_nodes"] = same / k
        prec["chord_error_rel"] = {"median": float(np.median(d)), "p99": float(np.percentile(d, 99)),
                                   "max": float(d.max())}
        c.set_x0(x_true.astype(np.float32))
        yk = c.project(0, k).cpu().numpy().astype(np.float64)
    with P.Context(g, n_blocks=40, flags=P.FLAG_NO_KAHAN, device=local) as c:
        c.load(S.subset(sub, slice(0, k)))
        c.set_x0(x_true.astype(np.float32))
        yp = c.project(0, k).cpu().numpy().astype(np.float64)
    y32 = O.project(g, S.subset(sub, slice(0, k)), x_true, mode=O.MODE_FP32)
    y64 = O.project(g, S.subset(sub, slice(0, k)), x_true, mode=O.MODE_FP64)
    m = y32 > 1.0
    prec["ax_rel_error_vs_fp64_sum_same_rows"] = {
        "kahan": {"max": float(np.max(np.abs(yk - y32)[m] / y32[m])), "mean": float(np.mean(np.abs(yk - y32)[m] / y32[m]))},
        "plain": {"max": float(np.max(np.abs(yp - y32)[m] / y32[m])), "mean": float(np.mean(np.abs(yp - y32)[m] / y32[m]))}}
    e64 = np.abs(yk - y64)[m] / y64[m]
    prec["ax_rel_error_vs_fp64_oracle"] = {"max": float(e64.max()), "mean": float(e64.mean()),
                                           "p99": float(np.percentile(e64, 99)),
                                           "p999": float(np.percentile(e64, 99.9))}
    with P.Context(g, n_blocks=40, device=local) as c:
        c.load(sub)
        c.iterate(wl.n_sweeps)
        xg = c.get_rsp().astype(np.float64)
    t0 = time.perf_counter()
    xo = O.drop_threads(g, sub, 40, wl.n_sweeps, mode=O.MODE_FP64)
    t_or = time.perf_counter() - t0
    rel = np.abs(xg - xo) / np.maximum(np.abs(xo), 1.0)
    roi = S.interior_mask(x_true, g)
    prec["rsp_error_vs_fp64_oracle"] = {"max": float(rel.max()), "mean": float(rel.mean()),
                                        "p999": float(np.percentile(rel, 99.9)), "bar": 1e-3,
                                        "roi_max": float(rel[roi].max()), "roi_mean": float(rel[roi].mean()),
                                        "note": "all voxels include sparsely sampled ones where a single index-list "
                                                "difference between FP32 and FP64 nodes decides the update"}
    prec["mean_rsp_error_vs_truth"] = {"gpu": S.mean_rsp_error(xg, x_true, g), "oracle": S.mean_rsp_error(xo, x_true, g)}
    prec["oracle_seconds"] = t_or
    return prec


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--subset", type=int, default=1_000_000, help="histories of the subset")
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args()
    print(json.dumps({"workload": "head160_precision_250000000", "precision": report(a.subset, a.device)}),
          flush=True)
