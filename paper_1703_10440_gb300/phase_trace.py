"""Per-phase timing of the MGS sweep kernel (CTA 0, %globaltimer).

Builds a copy of libmgsa with -DMGSA_PHASE_TRACE into ``_build/trace/`` (the
product library is left alone), runs a few QRs of each MGS form on one
workload and prints, per phase of the step loop, the mean time per step and
the total over the QR.  The traced kernel records at these points:

    step slot 0   step start
              1   norm partial of column i stored (HP: after the L update;
                  HA / naive: after the z_i update, its barrier and the MV)
              2   norm barrier passed (one-cluster launches: the window
                  holds the reduction of the rest of row i-1; whole-GPU
                  launches reload that row from R after it)
              3   r_ii formed (diagonal)
              4   pivots q_i, p_i formed (naive: after the second MV and its
                  barrier)
              5   main loop of the fused update/dot pass done
              6   warp pieces of the row partials combined
              7   CTA partials stored
              8   row barrier passed
              9   r_{i,i+1} summed (whole-GPU launches: and this CTA's share
                  of the rest of row i)

When a CTA's rows exceed one pivot chunk (staged mode), slots 4 and 5 are
recorded once per chunk and the last chunk's times remain: "pivots" then
also holds the fused passes of the earlier chunks.

Usage: python -m paper_1703_10440_gb300.phase_trace [poisson2d|varcoef3d|tridiag|denseband]
Needs a GPU.  Diagnostic only: the product build has no trace code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

from . import build as _build

PHASES = [(0, 1, "norm partial"), (1, 2, "norm barrier"), (2, 3, "diagonal"), (3, 4, "pivots"),
          (4, 5, "fused pass"), (5, 6, "combine pieces"), (6, 7, "store partials"), (7, 8, "row barrier"),
          (8, 9, "r_{i,i+1}")]


def build_traced() -> str:
    out_dir = os.path.join(_build.OUT_DIR, "trace")
    os.makedirs(out_dir, exist_ok=True)
    objs, procs = [], []
    for src in _build.sources():
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [_build.nvcc(), *_build.ARCH, *_build.NVCC_FLAGS, "-DMGSA_PHASE_TRACE", "-c", src, "-o", obj]
        procs.append(subprocess.Popen(cmd))
    if not all(p.wait() == 0 for p in procs):
        raise RuntimeError("nvcc failed on the traced build")
    lib = os.path.join(out_dir, "libmgsa_trace.so")
    subprocess.run([_build.nvcc(), *_build.ARCH, "-shared", "-cudart", "shared", "-o", lib, *objs], check=True)
    return lib


def main(argv: list[str]) -> None:
    which = argv[1] if len(argv) > 1 else "poisson2d"
    lib_path = build_traced()
    _build.LIB = lib_path  # load the traced copy instead of the product library
    import torch

    import workloads as W

    from . import mgsa

    gens = {"poisson2d": W.poisson2d, "varcoef3d": W.varcoef3d, "tridiag": lambda: W.tridiag(4096, 16),
            "denseband": W.denseband}
    A, Z = gens[which]()
    dev = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in A)
    Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev).T
    m, n = Z.shape
    L = mgsa.lib()
    L.mgsa_trace_fetch.restype = ctypes.c_int
    L.mgsa_trace_fetch.argtypes = [ctypes.c_void_p]
    buf = np.zeros((4200, 16), dtype=np.uint64)
    print(f"workload {which}: m = {m}, n = {n}, nnz = {len(A[1])}")
    with mgsa.Handle(0) as h:
        for v in ("naive", "ha", "hp"):
            for _ in range(3):
                h.qr(Ad, Zd, v)
                st = h.info()
                if st != (mgsa.MGSA_OK, 0):
                    raise RuntimeError(f"{v}: {st}")
            torch.cuda.synchronize()
            if L.mgsa_trace_fetch(buf.ctypes.data) != 0:
                raise RuntimeError("mgsa_trace_fetch failed")
            t = buf.astype(np.int64)
            T = t[: n - 1]  # the last step stops after its fused pass
            print(f"{v}: QR {(t[n - 1, 6] - t[4100, 0]) / 1e3:.1f} us, phase 0 {(t[4100, 1] - t[4100, 0]) / 1e3:.1f} us")
            print(f"  {'phase':16s} {'mean us/step':>12s} {'total us':>10s}")
            for a, b, name in PHASES:
                d = (T[:, b] - T[:, a]) / 1e3
                print(f"  {name:16s} {d.mean():12.2f} {d.sum():10.1f}")


if __name__ == "__main__":
    main(sys.argv)
