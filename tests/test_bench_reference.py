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
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] == d["e2e"]["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_single_instance():
    d = run("--workload", "tridiag")
    check_line(d)
    assert d["config"]["workload"] == "tridiag_m4096_n16"
    assert d["cpu_baseline"]["cores"] == bench_module().host_cores() or d["cpu_baseline"]["cores"] == 1


def bench_module():
    sys.path.insert(0, ROOT)
    import bench

    return bench


def test_default_workload_is_the_3d_laplacian():
    import argparse

    b = bench_module()
    seen = {}

    def fake_parse(self, *a, **k):
        seen.update({act.dest: act.default for act in self._actions})
        raise SystemExit(0)

    orig = argparse.ArgumentParser.parse_args
    argparse.ArgumentParser.parse_args = fake_parse
    try:
        try:
            b.main()
        except SystemExit:
            pass
    finally:
        argparse.ArgumentParser.parse_args = orig
    assert seen["workload"] == "varcoef3d" and seen["gpus"] == 1 and seen["warmup"] >= 3


def test_cpu_baseline_all_cores_and_single_thread():
    import workloads as W

    b = bench_module()
    A, Z = W.tridiag(3000, 12)
    cb = b.cpu_baseline(A, Z, "tridiag_m3000_n12")
    assert cb["kind"] == "oracle" and cb["unit"] == "QR/s" and cb["value"] > 0
    assert cb["cores"] >= 1 and str(cb["cores"]) in cb["sample"]
    st = cb["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and st["kind"] == "oracle"


def test_reference_batched_and_served():
    d = run("--workload", "batch4096", "--batch-count", "256")
    check_line(d)
    assert d["config"]["instances"] == 256
    d = run("--workload", "served")
    assert d == {"impl": "reference", "unavailable": d["unavailable"]} and d["unavailable"]


def test_derived_fp64_peak_from_sms_and_clock():
    b = bench_module()
    assert abs(b.derived_fp64_tflops(152, 2070.0) - 1.25856) < 1e-9  # 152 x 2 FMA/clk x 2 flop x 2.07 GHz
    assert b.derived_fp64_tflops(152, None) == b.derived_fp64_tflops(152, b.FALLBACK_SM_MHZ)
    assert abs(b.derived_fp64_tflops(76, 1000.0) - 0.304) < 1e-12
