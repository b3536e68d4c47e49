"""Write tests/golden/oracle_rows.json: regression values of the FP64 oracle.

Calls only oracle/ (and the seeded input generator). The inputs are stored
with the outputs, as float32 bit patterns, so the check does not depend on
the generator. Regenerate only with a change to the oracle's arithmetic that
names, in its commit message, the passage or reading that justifies it.

    python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1707_05014_gb300 import synthetic as S  # noqa: E402


def case(name, wl, count):
    g = wl.grid
    rec = S.subset(S.make_histories(wl), slice(0, count))
    out = {"name": name, "grid": [g.nx, g.ny, g.nz, g.hx, g.hy, g.hz],
           "records": {k: [int(b) for b in v.astype(np.float32).view(np.uint32)] for k, v in rec.items()},
           "table_nodes": None, "table": None}
    tab = O.mlp_table(g)
    nodes = sorted(set(range(0, len(tab), 8)) | {len(tab) - 1})
    out["table_nodes"], out["table"] = nodes, tab[nodes].tolist()
    for mode, tag in ((O.MODE_FP32, "fp32"), (O.MODE_FP64, "fp64")):
        rp, vox, ln = O.rows(g, rec, mode=mode)
        out[tag] = {"row_ptr": rp.tolist(), "vox": vox.tolist(), "len": ln.tolist()}
    out["project"] = O.project(g, rec, test_image(g.m)).tolist()
    x = O.drop(g, rec, 2, 2, mode=O.MODE_FP32)
    top = np.argsort(-np.abs(x), kind="stable")[:64]
    out["drop"] = {"blocks": 2, "sweeps": 2, "sum": float(x.sum()), "sumsq": float((x * x).sum()),
                   "top_index": top.tolist(), "top_value": x[top].tolist()}
    return out


def test_image(m):
    """A fixed image with no structure of its own: 1 + 0.001 (j mod 97)."""
    return 1.0 + 0.001 * (np.arange(m) % 97)


def main():
    cases = [case("water32", S.tiny_workload(16, seed=77), 16), case("head160", S.head_workload(4, seed=78), 4)]
    path = os.path.join(HERE, "oracle_rows.json")
    with open(path, "w") as f:
        json.dump({"about": "FP64 oracle regression values (rows in both node modes, MLP table, "
                            "a_i.x of a fixed image, 2 DROP sweeps summarised); inputs as float32 bit patterns; "
                            "written by tests/golden/make_oracle_golden.py",
                   "cases": cases}, f)
    print(path, os.path.getsize(path), "bytes")


if __name__ == "__main__":
    main()
