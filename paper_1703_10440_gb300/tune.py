"""Autotuner for libmgsa's launch parameters.

The kernels take a handful of launch parameters (``mgsa_set_param``): rows
per warp of the sparse products (one thread or one warp per CSR row), the
panel width of the block product X = A Z, the smallest row slab a CTA gets
(which sets the grid), the chunk of rows staged at once and, for batched
calls, the CTA count.  Which setting is fastest depends on the GPU, the form
of the method, the size of the problem and the density of A.  The tuner
times candidate settings on the actual problem with CUDA events, keeps the
fastest and caches it in a JSON file keyed by (GPU name, form, size bucket),
so later calls of the same shape reuse it.

Only launch parameters are searched; every candidate runs the same kernels
and gives results of the same accuracy (the row mode and the grid change the
reduction tree, the panel width and the batched CTA count change nothing).
"""
from __future__ import annotations

import itertools
import json
import math
import os

from . import mgsa

PARAMS = {
    "row_mode": mgsa.MGSA_PARAM_ROW_MODE,
    "spmm_panel": mgsa.MGSA_PARAM_SPMM_PANEL,
    "min_rows": mgsa.MGSA_PARAM_MIN_ROWS_PER_CTA,
    "chunk_rows": mgsa.MGSA_PARAM_CHUNK_ROWS,
    "batch_ctas": mgsa.MGSA_PARAM_BATCH_CTAS,
}

# Candidate values for one mgsa_qr call (0 = the library's default).
SINGLE_SPACE = {
    "row_mode": (1, 2),
    "spmm_panel": (4, 8),
    "min_rows": (32, 64, 128, 256),
    "chunk_rows": (0, 2048),
}

# Candidate values for one mgsa_qr_batched call.
BATCH_SPACE = {
    "row_mode": (1, 2),
    "spmm_panel": (4, 8),
}

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "mgsa", "tune.json")


def bucket_key(gpu: str, variant: str, m: int, n: int, nnz: int) -> str:
    """Shape bucket: m to the nearest power of two, n to the nearest multiple
    of 8, nonzeros per row to the nearest power of two."""
    mb = int(round(math.log2(max(m, 1))))
    nb = max(8, int(round(n / 8.0)) * 8)
    rb = int(round(math.log2(max(nnz / max(m, 1), 1.0))))
    return f"{gpu}|{variant}|m2^{mb}|n{nb}|nnz/row2^{rb}"


def candidates(space: dict, variant: str, rows_per_cta_max: int | None = None) -> list[dict]:
    """The grid of settings worth timing: the panel width only matters for
    the forms with a block product (HP), the chunk only when a CTA's slab can
    exceed one chunk."""
    keys = list(space)
    out = []
    for values in itertools.product(*(space[k] for k in keys)):
        c = dict(zip(keys, values))
        if "spmm_panel" in c and not variant.endswith("hp") and c["spmm_panel"] != 8:
            continue
        if "chunk_rows" in c and c["chunk_rows"] and rows_per_cta_max is not None and rows_per_cta_max <= c["chunk_rows"]:
            continue
        out.append(c)
    return out


def apply(handle: int, params: dict, set_param=None) -> None:
    """Set every parameter of ``params`` on the handle (others keep theirs)."""
    set_param = set_param or mgsa.mgsa_set_param
    for name, value in params.items():
        set_param(handle, PARAMS[name], int(value))


def reset(handle: int, names, set_param=None) -> None:
    """Give the named parameters their defaults back."""
    set_param = set_param or mgsa.mgsa_set_param
    for name in names:
        set_param(handle, PARAMS[name], 0)


class Tuner:
    """Times candidate settings and caches the fastest per shape bucket."""

    def __init__(self, path: str | None = None):
        self.path = path or os.environ.get("MGSA_TUNE_CACHE", DEFAULT_CACHE)
        self.cache: dict = {}
        if os.path.exists(self.path):
            with open(self.path) as f:
                self.cache = json.load(f)

    def save(self) -> None:
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def lookup(self, key: str) -> dict | None:
        hit = self.cache.get(key)
        return dict(hit["params"]) if hit else None

    def search(self, key: str, space: list[dict], time_fn, reps: int = 3) -> dict:
        """Time every candidate ``reps`` times with ``time_fn(params) -> ms``
        (the median counts), keep the fastest under ``key`` and return the
        record {"params", "ms", "trials"}."""
        trials = []
        for params in space:
            t = sorted(time_fn(params) for _ in range(reps))
            trials.append({"params": params, "ms": t[len(t) // 2]})
        best = min(trials, key=lambda x: x["ms"])
        rec = {"params": best["params"], "ms": best["ms"], "trials": trials}
        self.cache[key] = rec
        return rec

    # -- GPU-side drivers (time through the C ABI with CUDA events) --------

    def tune_qr(self, handle, A, Z, variant: str, reps: int = 3, warmup: int = 1) -> dict:
        """Tune mgsa_qr for (A, Z, variant) on ``handle`` (an ``mgsa.Handle``);
        returns the cache record and leaves the best setting applied."""
        import torch

        m, n = Z.shape
        nnz = A[1].numel()
        key = bucket_key(torch.cuda.get_device_name(Z.device), variant, m, n, nnz)
        sms = torch.cuda.get_device_properties(Z.device).multi_processor_count
        rows_max = (m + 31) // 32 * 32 if m < 32 * sms else None
        Q = torch.empty((n, m), dtype=torch.float64, device=Z.device).T
        R = torch.empty((n, n), dtype=torch.float64, device=Z.device).T
        names = list(SINGLE_SPACE)

        def time_fn(params):
            apply(handle.h, params)
            for _ in range(warmup):
                handle.qr_into(A, Z, Q, R, variant)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            handle.qr_into(A, Z, Q, R, variant)
            e1.record()
            e1.synchronize()
            st = handle.info()
            if st != (mgsa.MGSA_OK, 0):
                raise mgsa.MgsaError(st[0], f"candidate {params} failed with info {st[1]}")
            return e0.elapsed_time(e1)

        try:
            rec = self.search(key, candidates(SINGLE_SPACE, variant, rows_max), time_fn, reps)
        finally:
            reset(handle.h, names)
        apply(handle.h, rec["params"])
        return rec

    def tune_batched(self, handle, batch, reps: int = 3) -> dict:
        """Tune mgsa_qr_batched for a ``batch.Batch`` on ``handle`` (an
        ``mgsa.Handle``); the key uses the batch's largest instance."""
        import torch

        m = max(s[0] for s in batch.shapes)
        n = max(s[1] for s in batch.shapes)
        nnz = max(batch.nnz)
        key = bucket_key(torch.cuda.get_device_name(), "batched-" + "/".join(sorted(set(batch.variants))), m, n, nnz)
        names = list(BATCH_SPACE)
        variant = "hp" if "hp" in batch.variants else "ha"

        def time_fn(params):
            apply(handle.h, params)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            batch.run(handle.h)
            e1.record()
            e1.synchronize()
            return e0.elapsed_time(e1)

        try:
            rec = self.search(key, candidates(BATCH_SPACE, variant), time_fn, reps)
        finally:
            reset(handle.h, names)
        apply(handle.h, rec["params"])
        return rec
