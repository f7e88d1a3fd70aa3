"""Run a few QRs of one form on one named workload through the C ABI.

For profilers and quick checks: the same synthetic inputs as ``bench.py``
(seeded, built on the host, copied to the device once), then ``repeats``
calls of ``mgsa_qr`` on one stream, each followed by ``mgsa_get_info``.
Prints the CUDA-event time of every call.

Usage: python -m paper_1703_10440_gb300.run_once WORKLOAD FORM [REPEATS]
  WORKLOAD  poisson2d | varcoef3d | varcoef3d_64 | tridiag | denseband
            (varcoef3d_64: the 3D operator on a 64^3 grid with n = 128, an
            eighth of the rows of varcoef3d: inputs still larger than L2)
  FORM      naive | ha | hp | cgs_naive | cgs_ha | cgs_hp
"""
from __future__ import annotations

import sys

import numpy as np


def main(argv: list[str]) -> None:
    if len(argv) < 3:
        raise SystemExit(__doc__)
    which, form = argv[1], argv[2]
    repeats = int(argv[3]) if len(argv) > 3 else 2
    import torch

    import workloads as W

    from . import mgsa

    gens = {"poisson2d": W.poisson2d, "varcoef3d": W.varcoef3d, "varcoef3d_64": lambda: W.varcoef3d(side=64, n=128),
            "tridiag": lambda: W.tridiag(4096, 16),
            "denseband": W.denseband}
    if which not in gens or form not in mgsa.VARIANTS:
        raise SystemExit(__doc__)
    A, Z = gens[which]()
    dev = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in A)
    Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev).T
    m, n = Z.shape
    Q = torch.empty((n, m), dtype=torch.float64, device=dev).T
    R = torch.empty((n, n), dtype=torch.float64, device=dev).T
    stream = torch.cuda.current_stream(dev)
    with mgsa.Handle(0) as h:
        for k in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.qr_into(Ad, Zd, Q, R, form, stream)
            e1.record(stream)
            st = h.info(stream)
            if st != (mgsa.MGSA_OK, 0):
                raise SystemExit(f"{form} on {which}: status {st}")
            print(f"{which} m = {m} n = {n} {form}: call {k}: {e0.elapsed_time(e1):.3f} ms", flush=True)


if __name__ == "__main__":
    main(sys.argv)
