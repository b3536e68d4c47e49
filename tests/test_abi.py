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


def _lib_and_types():
    from paper_1707_05014_gb300 import build, pct

    lib = pct.load_library(build.build())
    return lib, pct


def _cfg(pct, **kw):
    c = dict(n_blocks=10, lam=1.0, node_step_mm=0.0, flags=0, clamp_min=0.0, threads_per_proton=1, cta_threads=128,
             tvs_beta0=0.0, tvs_alpha=0.99, tvs_eps=1e-4, tvs_tries=4, carp_strings=0)
    c.update(kw)
    return pct._Config(*c.values())


@pytest.mark.parametrize("grid,cfg,msg", [
    ((0, 32, 32, 2.0, 2.0, 2.0), {}, "grid dims"),
    ((600, 32, 32, 2.0, 2.0, 2.0), {}, "grid dims"),
    ((32, 32, 32, 0.0, 2.0, 2.0), {}, "voxel sizes"),
    ((32, 32, 32, 2.0, float("nan"), 2.0), {}, "voxel sizes"),
    ((32, 32, 32, 2.0, 2.0, 2.0), {"n_blocks": 0}, "n_blocks"),
    ((32, 32, 32, 2.0, 2.0, 2.0), {"lam": 2.0}, "lambda"),
    ((32, 32, 32, 2.0, 2.0, 2.0), {"threads_per_proton": 3}, "threads_per_proton"),
    ((32, 32, 32, 2.0, 2.0, 2.0), {"threads_per_proton": 64}, "threads_per_proton"),
    ((32, 32, 32, 2.0, 2.0, 2.0), {"node_step_mm": 1e-3}, "node count"),
    ((512, 512, 512, 1.0, 1.0, 1.0), {"node_step_mm": 100.0}, "fixed-point node range"),
])
def test_create_rejects_bad_arguments_before_touching_the_gpu(grid, cfg, msg):
    # Argument checks run on the host before any CUDA call, so they answer the
    # same with or without a GPU: PCT_ERR_INVALID_ARG, a message, no context.
    lib, pct = _lib_and_types()
    out = ctypes.c_void_p(123)
    rc = lib.pct_create(ctypes.byref(out), ctypes.byref(pct._Grid(*grid)), ctypes.byref(_cfg(pct, **cfg)), 0)
    assert rc == -1
    assert msg in lib.pct_last_error().decode()
    assert not out.value


def test_null_pointers_are_rejected():
    lib, pct = _lib_and_types()
    assert lib.pct_create(None, None, None, 0) == -1
    out = ctypes.c_void_p()
    assert lib.pct_create(ctypes.byref(out), None, None, 0) == -1
    assert lib.pct_measure_roofs(0, 0, None) == -1
    assert lib.pct_destroy(None) == 0  # NULL is a no-op
    lib.pct_drop_block_noalloc.argtypes = [ctypes.c_void_p] * 5
    assert lib.pct_drop_block_noalloc(None, None, None, None, None) == -1


@pytest.mark.parametrize("grid,n,lam,code,msg", [
    ((256, 256, 64, 1.0, 1.0, 1.0), 10, 1.0, -5, "fixed scratch"),  # 4.2M voxels > the 2,097,152 of the scratch
    ((128, 128, 128, 1.0, 1.0, 1.0), 10, 2.5, -1, "lambda"),  # exactly 2,097,152 voxels fit; lambda stops it next
    ((64, 64, 64, 1.0, 1.0, 1.0), 0, 1.0, -1, "n must be"),
    ((600, 64, 64, 1.0, 1.0, 1.0), 10, 1.0, -1, "grid dims"),
])
def test_no_alloc_update_checks_sizes_before_touching_the_gpu(grid, n, lam, code, msg):
    # The no-allocation block update validates the grid against its fixed
    # scratch and the history count on the host, before any CUDA call.
    lib, pct = _lib_and_types()
    lib.pct_drop_block_noalloc.argtypes = [ctypes.c_void_p] * 5
    g = pct._Grid(*grid)
    c = _cfg(pct, lam=lam)
    buf = (ctypes.c_float * 1)()
    h = pct._Hist(n, *([ctypes.addressof(buf)] * 11))
    rc = lib.pct_drop_block_noalloc(ctypes.byref(g), ctypes.byref(c), ctypes.byref(h), ctypes.addressof(buf), None)
    assert rc == code
    assert msg in lib.pct_last_error().decode()


def test_batch_and_network_arguments_are_checked_before_the_gpu():
    lib, pct = _lib_and_types()
    out = ctypes.c_void_p(7)
    assert lib.pct_batch_create(ctypes.byref(out), None, 0, None) == -1
    assert "at least one context" in lib.pct_last_error().decode() and not out.value
    for dims in ((8, 8, 12), (4, 8, 8), (0, 16, 16)):
        out = ctypes.c_void_p(7)
        assert lib.pct_net_create(ctypes.byref(out), *dims, 0, 0) == -1
        assert "multiples of 8" in lib.pct_last_error().decode() and not out.value


def test_header_is_plain_c_and_links_against_the_library(tmp_path):
    # A C (not C++) caller: include/pct.h compiles as C99 with warnings as
    # errors, and a program that takes the address of every declared entry
    # point links against libpct.so (names and C linkage agree).
    import shutil
    import subprocess

    from paper_1707_05014_gb300 import build

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    names = _declared("pct.h")
    src = tmp_path / "use_pct.c"
    src.write_text("#include \"pct.h\"\n#include <stdio.h>\nint main(void) {\n  void *p[] = {\n" +
                   ",\n".join(f"    (void *)&{n}" for n in names) +
                   "\n  };\n  printf(\"%d\\n\", (int)(sizeof p / sizeof p[0]));\n  return 0;\n}\n")
    exe = tmp_path / "use_pct"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", os.path.dirname(lib), "-lpct", f"-Wl,-rpath,{os.path.dirname(lib)}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and int(out.stdout) == len(names)


def test_shared_block_calls_check_arguments_before_the_gpu():
    lib, pct = _lib_and_types()
    assert lib.pct_block_partial(None, 0, None, None) == -1
    assert "NULL" in lib.pct_last_error().decode()
    assert lib.pct_block_apply(None, None, None) == -1
    assert "NULL" in lib.pct_last_error().decode()
    lib.pct_debug_fail_alloc(0)  # the testing hook is exported and disarms without a GPU
