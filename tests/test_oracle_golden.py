"""Regression check of the oracle against stored values
(tests/golden/oracle_rows.json, written by tests/golden/make_oracle_golden.py,
which calls only oracle/). Every pin elsewhere ties the oracle to the paper and
the mathematics; this one makes any later change to its arithmetic visible:
index lists and run counts must match exactly, floating-point values to the
last few bits."""
import json
import os

import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_rows.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("c", _cases(), ids=lambda c: c["name"])
def test_oracle_matches_its_stored_values(oracle, c):
    import importlib.util

    g = S.Grid(*c["grid"])
    rec = {k: np.array(v, dtype=np.uint32).view(np.float32) for k, v in c["records"].items()}
    tab = oracle.mlp_table(g)
    assert np.allclose(tab[c["table_nodes"]], np.array(c["table"]), rtol=1e-13, atol=1e-13)
    for mode, tag in ((oracle.MODE_FP32, "fp32"), (oracle.MODE_FP64, "fp64")):
        rp, vox, ln = oracle.rows(g, rec, mode=mode)
        assert rp.tolist() == c[tag]["row_ptr"]
        assert vox.tolist() == c[tag]["vox"]
        assert np.allclose(ln, np.array(c[tag]["len"]), rtol=1e-12, atol=0.0)
    spec = importlib.util.spec_from_file_location("make_oracle_golden", os.path.join(os.path.dirname(GOLDEN),
                                                                                       "make_oracle_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    assert np.allclose(oracle.project(g, rec, mk.test_image(g.m)), c["project"], rtol=1e-12, atol=0.0)
    d = c["drop"]
    x = oracle.drop(g, rec, d["blocks"], d["sweeps"], mode=oracle.MODE_FP32)
    assert np.isclose(x.sum(), d["sum"], rtol=1e-11) and np.isclose((x * x).sum(), d["sumsq"], rtol=1e-11)
    assert np.allclose(x[d["top_index"]], d["top_value"], rtol=1e-11, atol=1e-14)
