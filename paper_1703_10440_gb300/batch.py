"""Packing of many independent QR instances for ``mgsa_qr_batched``.

Argument marshalling only: the CSR arrays, Z, Q, R and the per-job
workspaces of all instances are packed into a handful of device buffers
(columns 256-byte aligned) and a device array of ``mgsa_job`` descriptors is
filled with pointers into them.  The QR itself runs in libmgsa's kernels.
"""
from __future__ import annotations

import numpy as np

from . import mgsa

# numpy mirror of mgsa_job (include/mgsa.h); 96 bytes.
JOB_DTYPE = np.dtype({
    "names": ["m", "n", "variant", "rowptr", "col", "val", "Z", "ldz", "Q", "ldq", "R", "ldr", "work"],
    "formats": ["<i8", "<i4", "<i4", "<u8", "<u8", "<u8", "<u8", "<i8", "<u8", "<i8", "<u8", "<i8", "<u8"],
    "offsets": [0, 8, 12, 16, 24, 32, 40, 48, 56, 64, 72, 80, 88],
    "itemsize": 96,
})
assert JOB_DTYPE.itemsize == __import__("ctypes").sizeof(mgsa.mgsa_job)

_ALIGN = 32  # elements: 256 bytes for doubles


def _round(x: int, q: int = _ALIGN) -> int:
    return (x + q - 1) // q * q


class Batch:
    """Device-resident batch.

    ``instances`` is a list of ``(A, Z)`` with ``A = (rowptr, col, val)`` numpy
    arrays and ``Z`` an ``m x n`` array; ``variants`` a list of variant names
    (or one name for all).  Jobs are laid out in the given order (put large
    instances first for the best load balance).
    """

    def __init__(self, instances, variants, device: int = 0):
        import torch

        self.torch = torch
        self.dev = torch.device("cuda", device)
        count = len(instances)
        if isinstance(variants, str):
            variants = [variants] * count
        self.count = count
        self.shapes = []
        self.nnz = [len(A[1]) for A, _ in instances]
        self.variants = [v if isinstance(v, str) else {i: k for k, i in mgsa.VARIANTS.items()}.get(int(v), str(v))
                         for v in variants]
        off_rp = off_col = off_val = off_z = off_r = off_w = 0
        layout = []
        for (A, Z), v in zip(instances, variants):
            rowptr, col, val = A
            m, n = Z.shape
            vi = mgsa.VARIANTS[v] if isinstance(v, str) else int(v)
            wbytes = mgsa.mgsa_job_workspace_bytes(m, n, vi) if vi in (0, 1, 2) else 8 * _round(m)
            layout.append((off_rp, off_col, off_val, off_z, off_r, off_w, m, n, vi))
            self.shapes.append((m, n))
            off_rp += _round(m + 1, 64)
            off_col += _round(max(len(col), 1), 64)
            off_val += _round(max(len(val), 1))
            off_z += _round(m) * n
            off_r += _round(n * n)
            off_w += _round(max(wbytes // 8, 1))
        t = torch
        self.rowptr = t.zeros(max(off_rp, 1), dtype=t.int32, device=self.dev)
        self.col = t.zeros(max(off_col, 1), dtype=t.int32, device=self.dev)
        self.val = t.zeros(max(off_val, 1), dtype=t.float64, device=self.dev)
        self.Z = t.zeros(max(off_z, 1), dtype=t.float64, device=self.dev)
        self.Q = t.zeros(max(off_z, 1), dtype=t.float64, device=self.dev)
        self.R = t.zeros(max(off_r, 1), dtype=t.float64, device=self.dev)
        self.work = t.zeros(max(off_w, 1), dtype=t.float64, device=self.dev)
        h_rp = np.zeros(self.rowptr.numel(), np.int32)
        h_col = np.zeros(self.col.numel(), np.int32)
        h_val = np.zeros(self.val.numel(), np.float64)
        h_z = np.zeros(self.Z.numel(), np.float64)
        jobs = np.zeros(count, dtype=JOB_DTYPE)
        self.offsets = []
        for k, ((A, Z), (orp, ocol, oval, oz, orr, ow, m, n, vi)) in enumerate(zip(instances, layout)):
            rowptr, col, val = A
            h_rp[orp:orp + m + 1] = rowptr
            h_col[ocol:ocol + len(col)] = col
            h_val[oval:oval + len(val)] = val
            ld = _round(m)
            h_z[oz: oz + ld * n].reshape(n, ld)[:, :m] = np.asarray(Z, dtype=np.float64).T
            jobs[k] = (m, n, vi, self.rowptr.data_ptr() + 4 * orp, self.col.data_ptr() + 4 * ocol,
                       self.val.data_ptr() + 8 * oval, self.Z.data_ptr() + 8 * oz, ld, self.Q.data_ptr() + 8 * oz,
                       ld, self.R.data_ptr() + 8 * orr, n, self.work.data_ptr() + 8 * ow)
            self.offsets.append((oz, ld, orr))
        self.rowptr.copy_(t.from_numpy(h_rp))
        self.col.copy_(t.from_numpy(h_col))
        self.val.copy_(t.from_numpy(h_val))
        self.Z.copy_(t.from_numpy(h_z))
        self.jobs_host = jobs
        self.jobs = t.from_numpy(jobs.view(np.uint8).copy()).to(self.dev)
        self.info = t.zeros(max(count, 1), dtype=t.int32, device=self.dev)

    def run(self, handle: int, stream=None) -> None:
        st = mgsa.mgsa_qr_batched(handle, self.count, self.jobs, self.info, stream)
        if st != mgsa.MGSA_OK:
            raise mgsa.MgsaError(st, mgsa.mgsa_last_error())

    def result(self, k: int):
        """(Q, R, info) of job k as numpy arrays (synchronises)."""
        m, n = self.shapes[k]
        oz, ld, orr = self.offsets[k]
        Q = self.Q[oz: oz + ld * n].view(n, ld)[:, :m].T.cpu().numpy()
        R = self.R[orr: orr + n * n].view(n, n).T.cpu().numpy()
        return Q, R, int(self.info[k].item())

    def infos(self) -> np.ndarray:
        return self.info[: self.count].cpu().numpy()
