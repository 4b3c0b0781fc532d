"""The reference arm of bench.py on the CPU: one JSON line with the contract's keys (the
GPU arm's line is exercised on the GPU by running bench.py itself)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    # the GPU arm's workload (the 8.04M-particle 3D dam break), each step a bounded sample
    assert line["config"]["workload"].startswith("3D dam break") and "dp = 1/159" in line["config"]["workload"]
    assert line["config"]["sample"]
    cb = line["cpu_baseline"]
    # every host core at once, one process each
    assert cb["kind"] == "oracle" and cb["cores"] == len(os.sched_getaffinity(0))
    assert cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
