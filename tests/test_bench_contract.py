"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the
JSON contract of the bench line; it needs no GPU. Under a launcher with several
ranks only rank 0 runs it."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--ref-sample", "3000"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    lines = _run({"RANK": "0", "OMP_NUM_THREADS": "2"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is True
    assert d["unit"] == "proton-iterations/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == 2 and "3000 histories" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    assert _run({"RANK": "1"}) == []


def test_clock_record_parses_nvidia_smi_samples():
    # The clocks object of the bench line: median SM clock under load, the
    # maximum, and every throttle reason seen Active (a run with hw_slowdown or
    # a thermal slowdown is rejected by the rules; sw_power_cap is kept).
    sys.path.insert(0, ROOT)
    import bench

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs._p = Done()
    cs.rows = [r.split(", ") for r in (
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    )]
    out = cs.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    cs.rows.append("0, 1500, 2070, 1000, 0x8, Active, Not Active, Active, Not Active".split(", "))
    assert cs.stop()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_counters_are_used_only_for_the_sources_they_were_taken_on(monkeypatch):
    # roofline.traffic comes from the committed ncu summary only while the
    # fused kernel's sources hash to the value recorded with it; otherwise null.
    sys.path.insert(0, ROOT)
    import bench

    with open(os.path.join(ROOT, "profiles", "drop_fused_head200_counters.json")) as f:
        rec = json.load(f)
    assert rec["sources"] == list(bench.FUSED_SOURCES) and rec["dram_bytes_per_history"] > 44
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["source_hash"])
    assert bench.ncu_counters()["dram_bytes_per_history"] == rec["dram_bytes_per_history"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_counters() is None


def test_source_hash_ignores_comments_and_layout_but_not_code():
    sys.path.insert(0, ROOT)
    import bench

    src = {f: "int f(int a) { return a + 1; }  // x\n" for f in bench.FUSED_SOURCES}
    h0 = bench.kernel_source_hash(src.__getitem__)
    commented = {f: "/* note */ int f(int a)\n{\n  return a + 1;  // y\n}\n" for f in bench.FUSED_SOURCES}
    assert bench.kernel_source_hash(commented.__getitem__) == h0
    changed = dict(src, **{bench.FUSED_SOURCES[0]: "int f(int a) { return a + 2; }"})
    assert bench.kernel_source_hash(changed.__getitem__) != h0
    assert bench.strip_c_comments('s = "//not a comment"; /* c */ t = 1; // c') == 's = "//not a comment"; t = 1;'


def test_traffic_is_reported_only_for_the_captured_configuration():
    sys.path.insert(0, ROOT)
    import argparse
    import bench

    with open(os.path.join(ROOT, "profiles", "drop_fused_head200_counters.json")) as f:
        rec = json.load(f)
    ok = argparse.Namespace(lanes=1, hull=False, workload=rec["workload"])
    n = rec["histories"]
    assert bench.traffic_per_launch(rec, ok, n) == rec["dram_bytes_per_history"] * n
    assert bench.traffic_per_launch(None, ok, n) is None
    assert bench.traffic_per_launch(rec, ok, n // 2) is None  # another launch size
    for bad in (dict(lanes=32), dict(hull=True), dict(workload="head")):
        assert bench.traffic_per_launch(rec, argparse.Namespace(**{**vars(ok), **bad}), n) is None


def test_oracle_is_loaded_only_by_tests_smoke_and_the_cpu_legs():
    # The oracle is test infrastructure: the package never imports it, and
    # bench.py loads it in one function only, the timing of the CPU baseline and
    # of the reference arm (oracle_rate).
    import ast

    pkg = os.path.join(ROOT, "paper_1707_05014_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            assert "oracle" not in {a.name.split(".")[0] for n in ast.walk(ast.parse(open(os.path.join(pkg, name)).read()))
                                    if isinstance(n, ast.Import) for a in n.names}, name
            assert not any(isinstance(n, ast.ImportFrom) and (n.module or "").startswith("oracle")
                           for n in ast.walk(ast.parse(open(os.path.join(pkg, name)).read()))), name
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    users = set()
    for f in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)]:
        for n in ast.walk(f):
            if isinstance(n, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in n.names):
                users.add(f.name)
            if isinstance(n, ast.ImportFrom) and (n.module or "").startswith("oracle"):
                users.add(f.name)
    assert users == {"oracle_rate"}
    assert not any(isinstance(n, (ast.Import, ast.ImportFrom)) and "oracle" in ast.dump(n) for n in tree.body)
