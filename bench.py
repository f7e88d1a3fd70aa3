#!/usr/bin/env python
"""Benchmark: A-orthonormal MGS thin QRs per second on GB300.

One step is one pass of the whole hot path over one synthetic input: the
same Z is factored by the three forms of the method -- naive (2n MV), MGS-HA
(n MV) and MGS-HP (one block product) -- so a step is 3 QRs and covers the
block SpMM, the per-column SpMVs, the diagonal, the A-dot rows and both
rank-1 updates.  Each QR is one cooperative kernel launch of libmgsa.

Default workload: 3D 7-point variable-coefficient Laplacian on a 128^3 grid
(face coefficients from per-cell exp(N(0,1))) + 1e-3 I (m = 2097152, CSR
FP64) and Z = N(0,1) of 2097152 x 128.  Each QR is timed with CUDA events on
the stream it runs on; L2 is flushed (a 256 MiB write) before every timed QR
(the inputs are larger than L2 as well).  After the timed region the default
line also carries, each with its own clock sample:

* ``batched``: the 4096-instance batched workload (one mgsa_qr_batched call per
  form) against one mgsa_qr launch per instance;
* ``served``: the continuous-batching server at 25 and 100 requests/s (p50 /
  p99 latency and each sampled request's slowdown over its solo latency) and
  its throughput on the 2000 requests/s stream (arrival window shortened to
  ``--extras-serve-window`` seconds; ``--workload served`` runs the full one);
* ``fp64_probe``: the measured FP64 FMA rate of the GPU (mgsa_fp64_probe).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mgsa|reference]
                    [--workload varcoef3d|poisson2d|tridiag|denseband|batch4096|served]

``--workload batch4096`` measures the batched path instead: 4096 banded SPD
instances (m ~ logU[256, 8192], n ~ U{4..64}) factored by one
mgsa_qr_batched call per variant, against one mgsa_qr launch per instance.

``--workload served`` runs the continuous-batching server on a Poisson stream
of requests (default 2000/s for 30 s; --serve-rate / --serve-seconds change
it and are reported in the line) and reports p50 / p99 latency and QRs/s;
--serve-sweep R1,R2,... serves the stream at several rates and reports each
sampled request's latency over its own solo latency.

``--impl reference`` times the CPU oracle on the host's cores on the same
workload: each step is one QR by the oracle's multi-core build (the same
operations and bits as the single-thread oracle, spread over all cores), the
forms taking turns; the batched workload runs sampled instances in one
single-thread oracle process per core.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "A-MGS QRs/sec & % HBM roofline (n-MV vs 2n-MV); served p50/p99 latency"
UNIT = "QR/s"
VARIANTS = ("naive", "ha", "hp")
L2_FLUSH_BYTES = 256 << 20
# Peaks: the measured HBM copy bandwidth (MEASURED_PEAKS.json), and for FP64
# the rate derived from unit counts and clocks -- SMs (device attribute) x 2
# FP64 FMA per clock x 2 flop x the SM clock sampled during the timed region --
# beside the rate the mgsa_fp64_probe kernel measures in the same run.
FP64_FMA_PER_CLK_SM = 2
FALLBACK_HBM_GBS = 6800.0
FALLBACK_SM_MHZ = 2070.0


def derived_fp64_tflops(sms: int, sm_mhz: float | None) -> float:
    return sms * FP64_FMA_PER_CLK_SM * 2 * (sm_mhz or FALLBACK_SM_MHZ) * 1e6 / 1e12
KERNEL_SOURCES = ["paper_1703_10440_gb300/csrc/mgsa_sweep.cu", "paper_1703_10440_gb300/csrc/mgsa_internal.cuh",
                  "paper_1703_10440_gb300/csrc/mgsa_device.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")


# ---------------------------------------------------------------------------
# Workloads and the algorithmic byte / flop models of each form
# ---------------------------------------------------------------------------

def make_workload(name: str):
    if name == "poisson2d":
        A, Z = W.poisson2d()
        desc = "poisson2d_512x512_shift0.01_n64_kappaZ1e6"
    elif name == "varcoef3d":
        A, Z = W.varcoef3d()
        desc = "varcoef3d_128cubed_shift1e-3_n128"
    elif name == "tridiag":
        A, Z = W.tridiag()
        desc = "tridiag_m4096_n16"
    elif name == "denseband":
        A, Z = W.denseband()
        desc = "denseband_m9180_hb194_n50_nnz3.5e6"
    else:
        raise SystemExit(f"unknown workload {name}")
    return desc, A, Z


def model(variant: str, m: int, n: int, nnz: int) -> tuple[float, float]:
    """Algorithmic (bytes, flops) of one QR in the right-looking one-pass-per-step form.

    c = 8m bytes per column, B_A = 12 nnz + 4(m+1) bytes of CSR.
    bytes  naive: 2n(B_A + 2c) + c n(n-1) + 2cn   (2n MV; z_j read+written per pair)
           HA:     n(B_A + 2c) + c n(n-1) + 2cn   (n MV)
           HP:     B_A + 2cn + 2c n(n-1) + 2cn    (one block product; z_j and x_j per pair)
    flops  per pair (i<j): dot + z-update (2 flop each per row), HP also x-update;
           per column: z^T x (2m), scaling by 1/r_ii (m per vector); MV 2 nnz.
    """
    c = 8.0 * m
    BA = 12.0 * nnz + 4.0 * (m + 1)
    pairs = n * (n - 1) / 2.0
    if variant == "naive":
        return 2 * n * (BA + 2 * c) + c * n * (n - 1) + 2 * c * n, 4.0 * m * pairs + 2.0 * m * n + m * n + 4.0 * nnz * n
    if variant == "ha":
        return n * (BA + 2 * c) + c * n * (n - 1) + 2 * c * n, 4.0 * m * pairs + 2.0 * m * n + 2.0 * m * n + 2.0 * nnz * n
    return BA + 2 * c * n + 2 * c * n * (n - 1) + 2 * c * n, 6.0 * m * pairs + 2.0 * m * n + 2.0 * m * n + 2.0 * nnz * n


def hbm_peak() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def read_traffic(workload: str, variant: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source."""
    try:
        rows = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 4 and not line.startswith("#"):
                    rows[(parts[0], parts[1])] = (parts[2], float(parts[3]))
        src, val = rows[(workload, variant)]
        return val if src == kernel_source_hash() else None
    except Exception:
        return None


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self) -> dict:
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and the reference arm)
# ---------------------------------------------------------------------------

def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(A, Z, variants, threads: int) -> tuple[float, int]:
    """Seconds for one oracle QR per form in ``variants`` by the multi-core
    build on ``threads`` threads (the same bits as the single-thread oracle),
    and the thread count it actually used."""
    import oracle

    used = oracle.par_threads(threads)
    t0 = time.perf_counter()
    for v in variants:
        _, _, info, _ = oracle.mgs_par(A, Z, v)
        if info != 0:
            raise RuntimeError(f"oracle breakdown in {v}")
    return time.perf_counter() - t0, used


def time_oracle_single(A, Z, variant) -> float:
    """Seconds for one QR by the single-thread oracle (plain C, row form)."""
    import oracle

    oracle.load()
    t0 = time.perf_counter()
    _, _, info, _, _ = oracle.mgs(A, Z, variant, "row")
    if info != 0:
        raise RuntimeError(f"oracle breakdown in {variant}")
    return time.perf_counter() - t0


def cpu_baseline(A, Z, desc, single_variant: str = "ha") -> dict:
    """The oracle timed on this host's cores: one QR per form by the multi-core
    build on every core (the headline CPU figure), and one QR by the
    single-thread oracle beside it."""
    cores = host_cores()
    secs, used = time_oracle(A, Z, VARIANTS, cores)
    one = time_oracle_single(A, Z, single_variant)
    return {"value": len(VARIANTS) / secs, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"one oracle QR per form (naive, ha, hp) of the same {desc} input by the oracle's multi-core "
                      f"build (row-form Algorithms 4/7/8, the single-thread oracle's operations and bits) on {used} "
                      f"threads: {len(VARIANTS)} QRs in {secs:.2f} s",
            "single_thread": {"value": 1.0 / one, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": f"one single-thread oracle QR (form {single_variant}, plain C FP64, row "
                                        f"form) of the same input: {one:.2f} s"}}


def run_reference(args, desc, A, Z, rank):
    if rank != 0:
        return
    m, n = Z.shape
    cores = host_cores()
    for k in range(args.warmup):
        time_oracle(A, Z, [VARIANTS[k % 3]], cores)
    secs, used = [], cores
    for k in range(args.steps):
        t, used = time_oracle(A, Z, [VARIANTS[k % 3]], cores)
        secs.append(t)
    total = sum(secs)
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "m": m, "n": n, "nnz": int(len(A[1])),
                       "step": "one QR, the forms naive/ha/hp taking turns"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"{args.steps} oracle QRs (multi-core build of the row-form Algorithms "
                                       f"4/7/8: the single-thread oracle's operations and bits) of the {desc} "
                                       f"workload on {used} threads, forms rotating"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


REF_BATCH_SAMPLE = 64  # instances per step of the batched workload's oracle arm


def _oracle_worker(task):
    """One single-thread oracle QR per instance (run in a worker process)."""
    instances, variant = task
    import oracle

    oracle.load()
    for A, Z in instances:
        _, _, info, _, _ = oracle.mgs(A, Z, variant, "row")
        if info != 0:
            raise RuntimeError(f"oracle breakdown in {variant}")
    return len(instances)


def run_reference_batch(args, rank):
    """Oracle arm of the batched workload: each step runs the single-thread
    oracle on a fixed sample of the batch's instances (one QR each, the forms
    taking turns by step), the instances spread over one process per core;
    QR/s over the sample."""
    if rank != 0:
        return
    import multiprocessing as mp

    inst = W.batch(args.batch_count)
    sample = inst[:: max(1, len(inst) // REF_BATCH_SAMPLE)][:REF_BATCH_SAMPLE]
    cores = min(host_cores(), len(sample))
    shards = [sample[c::cores] for c in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        def step(variant):
            t0 = time.perf_counter()
            done = sum(pool.map(_oracle_worker, [(sh, variant) for sh in shards]))
            assert done == len(sample)
            return time.perf_counter() - t0
        for k in range(args.warmup):
            step(VARIANTS[k % 3])
        secs = [step(VARIANTS[k % 3]) for k in range(args.steps)]
    total = sum(secs)
    value = len(sample) * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batch{len(inst)}_banded_hb8_m256-8192_n4-64", "instances": len(inst),
                       "step": f"one QR of each of {len(sample)} sampled instances, the forms taking turns by step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"every {max(1, len(inst) // REF_BATCH_SAMPLE)}-th instance of the batch "
                                       f"({len(sample)} of {len(inst)}), single-thread plain C FP64 oracle, "
                                       f"one process per core ({cores})"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def rank_reduce(x: float, op: str, world: int, device) -> float:
    """x combined over the ranks of the process group: "max" for times (the
    slowest rank sets the step), "sum" for throughputs.  Identity for one
    process.  ``device``: where the collective's tensor lives (CUDA for NCCL,
    CPU for gloo)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def fp64_probe(local_rank: int) -> dict:
    """The GPU's FP64 FMA rate measured by mgsa_fp64_probe, with the SM clock
    sampled while it ran."""
    from paper_1703_10440_gb300 import mgsa

    mgsa.mgsa_fp64_probe(local_rank, 2000)  # untimed: clocks up
    with ClockSampler(local_rank) as clk:
        best, ms = 0.0, 0.0
        for _ in range(5):
            tf, t = mgsa.mgsa_fp64_probe(local_rank, 40000)
            if tf > best:
                best, ms = tf, t
    return {"tflops": round(best, 4), "ms": round(ms, 3), "clocks": clk.summary(),
            "how": "mgsa_fp64_probe: 8 independent FMA chains per thread, 4 x 256 threads per SM, 40000 iterations, "
                   "best of 5 launches timed with CUDA events"}


def run_gpu(args, desc, A, Z, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1703_10440_gb300 import mgsa

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    m, n = Z.shape
    nnz = int(len(A[1]))
    rowptr, col, val = A
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (rowptr, col, val))
    Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev).T
    Q = torch.empty((n, m), dtype=torch.float64, device=dev).T
    R = torch.empty((n, n), dtype=torch.float64, device=dev).T
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    h = mgsa.Handle(local_rank)
    for v in VARIANTS:
        mgsa.mgsa_reserve(h.h, m, n, mgsa.VARIANTS[v])

    def one_qr(v):
        h.qr_into(Ad, Zd, Q, R, v, stream)

    for _ in range(args.warmup):
        for v in VARIANTS:
            flush.fill_(1)
            one_qr(v)
    st = h.info(stream)
    if st != (mgsa.MGSA_OK, 0):
        raise RuntimeError(f"warm-up QR failed: {st}")

    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in VARIANTS]
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            for vi, v in enumerate(VARIANTS):
                flush.fill_(k & 0xFF)
                ev[k][vi][0].record(stream)
                one_qr(v)
                ev[k][vi][1].record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    st = h.info(stream)
    if st != (mgsa.MGSA_OK, 0):
        raise RuntimeError(f"timed QR failed: {st}")
    per_variant_ms = [sum(ev[k][vi][0].elapsed_time(ev[k][vi][1]) for k in range(args.steps)) / args.steps
                      for vi in range(len(VARIANTS))]
    step_ms = sum(per_variant_ms)
    step_ms_max = rank_reduce(step_ms, "max", world, dev)
    clocks = clk.summary()

    # End to end through the host-buffer entry point: copies in, QR, copies out.
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        h_rp, h_col, h_val, h_Z = pin(rowptr), pin(col), pin(val), pin(np.asfortranarray(Z).T)
        h_Q = torch.empty((n, m), dtype=torch.float64).pin_memory()
        h_R = torch.empty((n, n), dtype=torch.float64).pin_memory()
        ksteps = max(3, min(args.steps, 10))

        def e2e_step():
            for v in VARIANTS:
                r = mgsa.mgsa_qr_host(h.h, h_rp, h_col, h_val, nnz, h_Z, m, n, m, mgsa.VARIANTS[v], h_Q, m, h_R, n,
                                      stream)
                if r != (mgsa.MGSA_OK, 0):
                    raise RuntimeError(f"mgsa_qr_host failed: {r}")
        e2e_step()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(ksteps):
            e2e_step()
        torch.cuda.synchronize(dev)
        e2e_ms = rank_reduce(1e3 * (time.perf_counter() - t0) / ksteps, "max", world, dev)
        h2d = 3 * (rowptr.nbytes + col.nbytes + val.nbytes + Z.nbytes)
        d2h = 3 * (8 * m * n + 8 * n * n)
        e2e = {"value": world * 3 * 1e3 / e2e_ms, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms, "steps": ksteps}
        del h_rp, h_col, h_val, h_Z, h_Q, h_R
    h.close()
    del Ad, Zd, Q, R
    torch.cuda.empty_cache()

    probe = fp64_probe(local_rank) if not args.no_extras else None
    extras = {}
    if not args.no_extras:
        extras["batched"] = measure_batch(args, local_rank, steps=min(args.steps, 5), warmup=3)
        extras["served"] = measure_served_summary(args, local_rank)

    if rank != 0:
        return
    peak_hbm, peak_src = hbm_peak()
    fp64_peak = derived_fp64_tflops(sms, clocks.get("sm_mhz"))
    per_variant = {}
    for vi, v in enumerate(VARIANTS):
        b, fl = model(v, m, n, nnz)
        ms = per_variant_ms[vi]
        gbs = b / ms / 1e6
        tfl = fl / ms / 1e9
        per_variant[v] = {"ms": round(ms, 4), "qr_per_s": round(1e3 / ms, 2), "cols_per_s": round(n * 1e3 / ms, 1),
                          "model_bytes": b, "model_flops": fl,
                          "model_GBs": round(gbs, 1), "hbm_frac": round(gbs / peak_hbm, 4),
                          "fp64_tflops": round(tfl, 4), "fp64_frac": round(tfl / fp64_peak, 4)}
        if probe:
            per_variant[v]["fp64_frac_of_probe"] = round(tfl / probe["tflops"], 4)
    # Dominant kernel: the longest of the three launches of a step.
    dom = max(VARIANTS, key=lambda v: per_variant[v]["ms"])
    pv = per_variant[dom]
    if pv["fp64_frac"] >= pv["hbm_frac"]:
        roof = {"bound": "alu", "achieved": pv["fp64_tflops"], "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                "frac": pv["fp64_frac"]}
    else:
        roof = {"bound": "hbm", "achieved": pv["model_GBs"], "peak": peak_hbm, "unit": "GB/s", "frac": pv["hbm_frac"]}
    traffic = read_traffic(desc, dom)
    roof.update({"traffic": traffic, "kernel": f"mgs_sweep_kernel<{dom}>",
                 "algorithmic_bytes": pv["model_bytes"], "algorithmic_flops": pv["model_flops"],
                 "hbm_achieved_GBs": pv["model_GBs"], "hbm_peak_GBs": peak_hbm,
                 "hbm_frac_of_" + peak_src: pv["hbm_frac"],
                 "fp64_peak_derived": {"tflops": round(fp64_peak, 4), "sms": sms,
                                       "fma_per_clk_per_sm": FP64_FMA_PER_CLK_SM,
                                       "sm_mhz": clocks.get("sm_mhz") or FALLBACK_SM_MHZ,
                                       "sm_mhz_source": "median sampled in the timed region"
                                       if clocks.get("sm_mhz") else "fallback (no clock samples)"},
                 "fp64_frac_of_derived_peak": pv["fp64_frac"]})
    if probe:
        roof["fp64_probe_tflops"] = probe["tflops"]
        roof["fp64_frac_of_probe"] = pv.get("fp64_frac_of_probe")

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(A, Z, desc)

    value = world * 3 * 1e3 / step_ms_max
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "m": m, "n": n, "nnz": nnz, "step": "3 QRs: naive, ha, hp on the same Z",
                       "l2": "flushed (256 MiB write) before every timed QR; inputs larger than L2",
                       "parallelism": f"replicas{world}"},
            "per_variant": per_variant, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 3 * args.steps, "clocks": clocks}
    if probe:
        line["fp64_probe"] = probe
    line.update(extras)
    print(json.dumps(line), flush=True)


def measure_batch(args, local_rank, steps: int, warmup: int) -> dict:
    """Batched path: one mgsa_qr_batched call per form over the 4096-instance
    workload, and one mgsa_qr launch per instance of the same HP jobs."""
    import torch

    from paper_1703_10440_gb300 import mgsa
    from paper_1703_10440_gb300.batch import Batch

    dev = torch.device("cuda", local_rank)
    inst = W.batch(args.batch_count)
    # largest work first for the queue's load balance
    order = sorted(range(len(inst)), key=lambda k: -inst[k][1].shape[0] * inst[k][1].shape[1] ** 2)
    inst = [inst[k] for k in order]
    batches = {v: Batch(inst, v, device=local_rank) for v in VARIANTS}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    h = mgsa.Handle(local_rank)
    for _ in range(warmup):
        for v in VARIANTS:
            batches[v].run(h.h, stream)
    torch.cuda.synchronize(dev)
    for v in VARIANTS:
        bad = int((batches[v].infos() != 0).sum())
        if bad:
            raise RuntimeError(f"{bad} batched {v} jobs failed")
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in VARIANTS]
          for _ in range(steps)]
    torch.cuda.synchronize(dev)
    with ClockSampler(local_rank) as clk:
        for k in range(steps):
            for vi, v in enumerate(VARIANTS):
                flush.fill_(k & 0xFF)
                ev[k][vi][0].record(stream)
                batches[v].run(h.h, stream)
                ev[k][vi][1].record(stream)
        torch.cuda.synchronize(dev)
    per_ms = [sum(ev[k][vi][0].elapsed_time(ev[k][vi][1]) for k in range(steps)) / steps
              for vi in range(len(VARIANTS))]
    # One launch per instance (the single-instance entry point), same inputs.
    single_ms = {}
    for v in ("hp",):
        b = batches[v]
        csrs = []
        for k in range(b.count):
            j = b.jobs_host[k]
            csrs.append((mgsa.make_csr(int(j["m"]), 0, int(j["rowptr"]), int(j["col"]), int(j["val"])), j))

        def per_instance():
            for csr, j in csrs:
                st = mgsa.mgsa_qr(h.h, csr, int(j["Z"]), int(j["m"]), int(j["n"]), int(j["ldz"]), mgsa.VARIANTS[v],
                                  int(j["Q"]), int(j["ldq"]), int(j["R"]), int(j["ldr"]), stream)
                if st != mgsa.MGSA_OK:
                    raise RuntimeError(mgsa.mgsa_last_error())
        for csr, j in csrs:
            mgsa.mgsa_reserve(h.h, int(j["m"]), int(j["n"]), mgsa.VARIANTS[v])
        per_instance()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        per_instance()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        single_ms[v] = e0.elapsed_time(e1)
    h.close()
    del batches
    torch.cuda.empty_cache()
    ms_sizes = [Z.shape for _, Z in inst]
    nnz = [len(A[1]) for A, _ in inst]
    per_variant = {}
    for vi, v in enumerate(VARIANTS):
        fl = sum(model(v, m, n, z)[1] for (m, n), z in zip(ms_sizes, nnz))
        tfl = fl / per_ms[vi] / 1e9
        per_variant[v] = {"ms": round(per_ms[vi], 3), "qr_per_s": round(len(inst) * 1e3 / per_ms[vi], 1),
                          "cols_per_s": round(sum(n for _, n in ms_sizes) * 1e3 / per_ms[vi], 1),
                          "model_flops": fl, "fp64_tflops": round(tfl, 4)}
    clocks = clk.summary()
    return {"workload": f"batch{len(inst)}_banded_hb8_m256-8192_n4-64", "instances": len(inst),
            "steps": steps, "warmup": warmup, "per_variant": per_variant, "total_ms": sum(per_ms),
            "one_launch_per_instance": {v: {"ms": round(t, 3), "qr_per_s": round(len(inst) * 1e3 / t, 1),
                                            "batched_speedup": round(t / per_variant[v]["ms"], 2)}
                                        for v, t in single_ms.items()},
            "gpu_launches": 9 * steps, "clocks": clocks,
            "fp64_peak_derived_tflops": round(derived_fp64_tflops(
                torch.cuda.get_device_properties(dev).multi_processor_count, clocks.get("sm_mhz")), 4)}


def run_batch(args, rank, world, local_rank):
    """Batched workload line: one mgsa_qr_batched call per form over 4096
    instances per step."""
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.barrier()
    res = measure_batch(args, local_rank, args.steps, args.warmup)
    step_ms_max = rank_reduce(res["total_ms"], "max", world, dev)
    if rank != 0:
        return
    peak = res["fp64_peak_derived_tflops"]
    for pv in res["per_variant"].values():
        pv["fp64_frac"] = round(pv["fp64_tflops"] / peak, 4)
    dom = max(VARIANTS, key=lambda v: res["per_variant"][v]["ms"])
    pv = res["per_variant"][dom]
    line = {"metric": METRIC, "value": world * 3 * res["instances"] * 1e3 / step_ms_max, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": res["workload"], "instances": res["instances"],
                       "step": "one mgsa_qr_batched call per variant (naive, ha, hp)",
                       "l2": "flushed (256 MiB write) before every timed call", "parallelism": f"replicas{world}"},
            "per_variant": res["per_variant"],
            "roofline": {"bound": "alu", "achieved": pv["fp64_tflops"], "peak": peak, "unit": "TFLOP/s",
                         "frac": pv["fp64_frac"], "traffic": None, "kernel": f"mgs_batch_kernel<{dom}>"},
            "one_launch_per_instance": res["one_launch_per_instance"],
            "gpu_launches": res["gpu_launches"], "clocks": res["clocks"]}
    print(json.dumps(line), flush=True)


def serve_runs(args, local_rank, rank, rates, seconds, sample_size):
    """Serve the Poisson stream at each rate in turn; returns the per-rate
    statistics, each sampled request's slowdown over its solo latency, and
    the solo latencies."""
    import torch

    from paper_1703_10440_gb300 import mgsa
    from paper_1703_10440_gb300.serve import Request, Server, poisson_arrivals

    torch.cuda.set_device(local_rank)
    h = mgsa.Handle(local_rank)
    srv = Server(h.h, args.serve_variant, budget_bytes=120e9, small_work=args.serve_small_work, device=local_rank,
                 small_ctas=args.serve_small_ctas, max_large_inflight=args.serve_large_window,
                 slice_ms=args.serve_slice_ms, large_mode=args.serve_large_mode, admit_per_tick=args.serve_admit_per_tick,
                 small_variant=args.serve_small_variant or None)
    streams = {(rate, secs): poisson_arrivals(rate, secs, seed=W.SEED + rank) for rate, secs in zip(rates, seconds)}
    first = streams[(rates[0], seconds[0])]
    srv.run([Request(10**7 + k, r.m, r.n, r.kind, 0.0, r.seed) for k, r in enumerate(first[:4])], realtime=False)
    g = np.random.Generator(np.random.PCG64(7))
    runs = []
    with ClockSampler(local_rank) as clk:
        for rate, secs in zip(rates, seconds):
            reqs = streams[(rate, secs)]
            stats = srv.run(reqs, realtime=True)
            lat = dict(srv.last_latency_s)
            k = min(sample_size, len(reqs))
            sample = sorted(g.choice(len(reqs), size=k, replace=False).tolist()) if k else []
            runs.append((rate, secs, reqs, stats, lat, sample))
    # solo latency of every sampled request (sizes depend only on the index)
    by_rid = {}
    for _, _, reqs, _, _, sample in runs:
        for k in sample:
            by_rid.setdefault(reqs[k].rid, reqs[k])
    solo = {}
    for rid, r in sorted(by_rid.items()):
        srv.run([Request(r.rid, r.m, r.n, r.kind, 0.0, r.seed)], realtime=False)
        solo[rid] = srv.last_latency_s[rid]
    srv.close()
    h.close()
    sweep = []
    for rate, secs, reqs, stats, lat, sample in runs:
        slow = np.array([lat[reqs[k].rid] / solo[reqs[k].rid] for k in sample]) if sample else np.array([np.nan])
        sweep.append({"rate_per_s": rate, "seconds": secs, "requests": stats["requests"], "ok": stats["ok"],
                      "qr_per_s": stats["qr_per_s"], "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"],
                      "p50_slowdown": float(np.percentile(slow, 50)), "p99_slowdown": float(np.percentile(slow, 99)),
                      "slowdown_sample": len(sample), "launches": stats["launches"], "small": stats["small"],
                      "peak_bytes": stats["peak_bytes"], "makespan_s": stats["makespan_s"]})
    solo_s = np.array(list(solo.values())) if solo else np.array([np.nan])
    solo_p99_ms = float(np.percentile(solo_s, 99) * 1e3)
    for x in sweep:
        x["p99_over_solo_p99"] = x["p99_ms"] / solo_p99_ms
    return sweep, solo_s, clk.summary()


def measure_served_summary(args, local_rank) -> dict:
    """The served numbers carried by the default line: p50 / p99 latency and
    the per-request p99 slowdown at 25 and 100 requests/s (10 s each), and
    QR/s on the 2000 requests/s stream with a shortened arrival window."""
    rates = [25.0, 100.0, 2000.0]
    seconds = [10.0, 10.0, args.extras_serve_window]
    sweep, solo_s, clocks = serve_runs(args, local_rank, 0, rates, seconds, sample_size=100)
    sweep[-1]["slowdown_sample"] = 0  # not sampled: the point of that run is throughput under a backlog
    for key in ("p50_slowdown", "p99_slowdown", "p99_over_solo_p99"):
        sweep[-1].pop(key, None)
    return {"workload": "served_poisson_m1e3-1e6_n8-128_laplace/banded", "variant": args.serve_variant,
            "small_variant": args.serve_small_variant or args.serve_variant,
            "budget_gb": 120, "large_mode": args.serve_large_mode, "slice_ms": args.serve_slice_ms,
            "large_window": args.serve_large_window, "sweep": sweep, "solo_p50_ms": float(np.median(solo_s) * 1e3),
            "solo_p99_ms": float(np.percentile(solo_s, 99) * 1e3),
            "qr_per_s_at_2000_per_s": sweep[-1]["qr_per_s"],
            "note": f"the 2000 req/s stream arrives for {args.extras_serve_window:g} s here (30 s under "
                    f"--workload served); slowdown = latency / the same request's latency alone on an idle GPU",
            "clocks": clocks, "gpu_launches": int(sum(x["launches"] for x in sweep))}


def run_served(args, rank, world, local_rank):
    """Served stream: Poisson arrivals (default 2000/s for 30 s), m ~ logU[1e3, 1e6],
    n ~ U{8..128}, 50/50 Laplacian / banded, 120 GB admission budget.

    With --serve-sweep R1,R2,... the stream is served at each rate in turn and
    every sampled request's latency is divided by its own solo latency (the
    same request served alone on an idle GPU); the line reports, per rate,
    p50 / p99 latency, p99 of that slowdown and QR/s, the largest rate whose
    p99 slowdown is at most 2, and serving against one solo call at a time."""
    import torch

    rates = [float(x) for x in args.serve_sweep.split(",")] if args.serve_sweep else [args.serve_rate]
    sweep, solo_s, clocks = serve_runs(args, local_rank, rank, rates, [args.serve_seconds] * len(rates),
                                       args.serve_sample)
    total_qr_per_s = rank_reduce(sweep[-1]["qr_per_s"], "sum", world, torch.device("cuda", local_rank))
    if rank != 0:
        return
    serial_qr_per_s = len(solo_s) / float(solo_s.sum())
    ok_rates = [x["rate_per_s"] for x in sweep if x["p99_slowdown"] <= 2.0]
    ok_rates_dist = [x["rate_per_s"] for x in sweep if x["p99_over_solo_p99"] <= 2.0]
    main = sweep[-1]
    line = {"metric": METRIC, "value": total_qr_per_s, "unit": UNIT, "n_gpus": world, "steps": 1,
            "warmup": 1, "ms_per_step": main["makespan_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "served_poisson_m1e3-1e6_n8-128_laplace/banded", "rate_per_s": main["rate_per_s"],
                       "seconds": args.serve_seconds, "requests": main["requests"], "variant": args.serve_variant,
                       "small_variant": args.serve_small_variant or args.serve_variant,
                       "budget_gb": 120, "small_work": args.serve_small_work, "small_ctas": args.serve_small_ctas,
                       "large_window": args.serve_large_window, "slice_ms": args.serve_slice_ms,
                       "large_mode": args.serve_large_mode, "admit_per_tick": args.serve_admit_per_tick},
            "served": {"sweep": sweep, "solo_p50_ms": float(np.median(solo_s) * 1e3),
                       "solo_p99_ms": float(np.percentile(solo_s, 99) * 1e3),
                       "solo_serial_qr_per_s": serial_qr_per_s,
                       "served_over_serial": main["qr_per_s"] / serial_qr_per_s,
                       "max_rate_p99_slowdown_le_2": max(ok_rates) if ok_rates else None,
                       "max_rate_p99_le_2x_solo_p99": max(ok_rates_dist) if ok_rates_dist else None},
            "gpu_launches": int(sum(x["launches"] for x in sweep)), "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mgsa", choices=["mgsa", "reference"])
    ap.add_argument("--workload", default="varcoef3d",
                    choices=["varcoef3d", "poisson2d", "tridiag", "denseband", "batch4096", "served"])
    ap.add_argument("--batch-count", type=int, default=4096,
                    help="batch4096: instances per batched call (4096 is the workload; fewer for profiling)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="served: arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=30.0, help="served: arrival window")
    ap.add_argument("--serve-variant", default="ha", choices=["naive", "ha", "hp"],
                    help="served: form of the requests (HA: the fastest form on the served matrices)")
    ap.add_argument("--serve-small-variant", default="", choices=["", "naive", "ha", "hp"],
                    help="served: form of the small (batched) requests; default: --serve-variant")
    ap.add_argument("--serve-small-work", type=float, default=2e7, help="served: m*n^2 up to which the batched kernel runs")
    ap.add_argument("--serve-sweep", default="", help="served: comma-separated arrival rates run in turn")
    ap.add_argument("--serve-sample", type=int, default=200, help="served: requests per rate timed alone as well")
    ap.add_argument("--serve-small-ctas", type=int, default=16,
                    help="served: SMs kept for small requests (0 = no partition)")
    ap.add_argument("--serve-large-window", type=int, default=2,
                    help="served: large launches kept in flight, least work first (0 = all, in arrival order)")
    ap.add_argument("--serve-slice-ms", type=float, default=2.0,
                    help="served: time slices of about this long for large requests (0 = whole QRs)")
    ap.add_argument("--serve-large-mode", default="group", choices=["group", "slices"],
                    help="served: time slices of large requests as grouped launches (gangs of CTAs side by side) "
                         "or as whole-GPU launches of one request each")
    ap.add_argument("--serve-admit-per-tick", type=int, default=16,
                    help="served: requests admitted (inputs drawn) per turn of the serving loop (0 = no limit)")
    ap.add_argument("--extras-serve-window", type=float, default=2.0,
                    help="default line: arrival window (s) of the 2000 req/s stream in the served key")
    ap.add_argument("--no-extras", action="store_true",
                    help="single-instance workloads: skip the batched / served / fp64_probe keys")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        if args.workload == "batch4096":
            run_reference_batch(args, rank)
        elif args.workload == "served":
            print(json.dumps({"impl": "reference", "unavailable": "the served stream's inputs are drawn on the GPU at "
                                                                  "admission; the oracle arm covers the single-instance "
                                                                  "and batched workloads"}), flush=True)
        else:
            desc, A, Z = make_workload(args.workload)
            run_reference(args, desc, A, Z, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.workload == "batch4096":
        run_batch(args, rank, world, local_rank)
    elif args.workload == "served":
        run_served(args, rank, world, local_rank)
    else:
        desc, A, Z = make_workload(args.workload)
        run_gpu(args, desc, A, Z, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
