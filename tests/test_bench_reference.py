"""bench.py's reference arm on the host (no GPU): the oracle as it stands, one copy per
host core, prints the contract's JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "4",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["steps"] == 4 and d["warmup"] == 3 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the same workload object as the GPU arm's line
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    assert d["config"] == bench.bench_config(W.config_binary_16384x256(), 1)
    assert d["metric"] == bench.METRIC


def test_bench_options():
    """The options the benchmark contract and the profiles' commands use."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True,
                         text=True, timeout=120, cwd=ROOT).stdout
    for opt in ("--gpus", "--steps", "--warmup", "--impl", "--tile", "--storage", "--profile", "--no-cpu-baseline",
                "--no-batch", "--no-surrogate", "--workload", "lg_16384x256", "f32b"):
        assert opt in out, opt
