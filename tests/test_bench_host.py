"""Host-side parts of bench.py that need no GPU: the reference arm's JSON line
(the FP64 oracle timed on the host cores), its behaviour on ranks other than 0,
and the rule that the ncu traffic figure is reported only for the kernel
sources it was captured from."""

import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=300)


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_reference_arm_line():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference"
    assert j["unit"] == "features/s" and j["higher_is_better"] is True
    assert j["value"] > 0 and j["steps"] == 1 and j["warmup"] == 1 and j["n_gpus"] == 1
    assert j["config"]["workload"] == "fastfood_features_rbf" and j["config"]["d"] == 1024
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
    assert j["cpu_baseline"]["value"] == j["value"] and j["cpu_baseline"]["sample"]
    assert j["e2e"] == {"value": j["value"], "unit": "features/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "1"],
             {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_traffic_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    b = _bench_module()
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        entry = json.load(f)["k_feat_warp<10,0>"]
    monkeypatch.setattr(b, "kernel_source_hash", lambda: entry["source_hash"])
    assert b.ncu_traffic("k_feat_warp<10,0>") == entry["dram_bytes_per_launch"]
    monkeypatch.setattr(b, "kernel_source_hash", lambda: "0" * 16)
    assert b.ncu_traffic("k_feat_warp<10,0>") is None
    assert b.ncu_traffic("no_such_kernel") is None
