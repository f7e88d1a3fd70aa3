"""The oracle arm of bench.py (``--impl reference``) on the CPU: one JSON
line with the contract's keys, for a single-instance workload and for the
batched one; the served workload reports itself unavailable."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2", "--warmup", "3",
           *extra]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def check_line(d):
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "QR/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"] == d["e2e"]["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_single_instance():
    d = run("--workload", "tridiag")
    check_line(d)
    assert d["config"]["workload"] == "tridiag_m4096_n16"


def test_reference_batched_and_served():
    d = run("--workload", "batch4096", "--batch-count", "256")
    check_line(d)
    assert d["config"]["instances"] == 256
    d = run("--workload", "served")
    assert d == {"impl": "reference", "unavailable": d["unavailable"]} and d["unavailable"]
