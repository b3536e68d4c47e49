"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/pct.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"^PCT_API\s+[\w\s\*]+?\b(pct_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared("pct.h")
    for required in ("pct_create", "pct_destroy", "pct_load_histories", "pct_mlp_rows", "pct_iterate",
                     "pct_get_rsp", "pct_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1707_05014_gb300 import build

    lib = ctypes.CDLL(build.build())
    headers = [h for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]
    for h in headers:
        for name in _declared(h):
            assert hasattr(lib, name), f"{name} declared in {h} but not exported"


def test_binding_refuses_to_run_without_library(tmp_path):
    from paper_1707_05014_gb300 import pct

    with pytest.raises(ImportError):
        pct.load_library(str(tmp_path / "missing.so"))


def test_last_error_is_reported_without_gpu():
    # argument validation happens before any CUDA call
    from paper_1707_05014_gb300 import pct

    L = pct.load_library()
    h = ctypes.c_void_p()
    g = pct._Grid(0, 4, 4, 1.0, 1.0, 1.0)
    c = pct._Config(1, 1.0, 0.0, 0, 0.0, 1, 128)
    assert L.pct_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(c), 0) == -1
    assert b"grid dims" in L.pct_last_error()
    g = pct._Grid(4, 4, 4, 1.0, 1.0, 1.0)
    c = pct._Config(1, 2.5, 0.0, 0, 0.0, 1, 128)
    assert L.pct_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(c), 0) == -1
    assert b"lambda" in L.pct_last_error()
