"""ctypes binding of libmgsa (declared in ``include/mgsa.h``).

Argument marshalling only: every step of the QR runs in the library's CUDA
kernels.  Functions keep the C names.  Device buffers are passed as raw
pointers (``int``) or as CUDA torch tensors (their ``data_ptr()``); PyTorch is
used for device memory and streams, nothing else.

If ``libmgsa.so`` is missing it is built in-tree with nvcc; if that is not
possible the import fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

MGSA_NAIVE, MGSA_HA, MGSA_HP = 0, 1, 2
MGSA_CGS_NAIVE, MGSA_CGS_HA, MGSA_CGS_HP = 3, 4, 5
VARIANTS = {"naive": MGSA_NAIVE, "ha": MGSA_HA, "hp": MGSA_HP,
            "cgs_naive": MGSA_CGS_NAIVE, "cgs_ha": MGSA_CGS_HA, "cgs_hp": MGSA_CGS_HP}

MGSA_OK = 0
MGSA_ERR_INVALID = 1
MGSA_ERR_BREAKDOWN = 2
MGSA_ERR_NONFINITE = 3
MGSA_ERR_NOMEM = 4
MGSA_ERR_CUDA = 5
MGSA_ERR_TIMEOUT = 6
STATUS_NAMES = {0: "MGSA_OK", 1: "MGSA_ERR_INVALID", 2: "MGSA_ERR_BREAKDOWN", 3: "MGSA_ERR_NONFINITE",
                4: "MGSA_ERR_NOMEM", 5: "MGSA_ERR_CUDA", 6: "MGSA_ERR_TIMEOUT"}
MGSA_MAX_N = 2048
MGSA_NOALLOC_SCRATCH_BYTES = 32 << 20


class mgsa_csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class mgsa_job(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("Z", ctypes.c_void_p), ("ldz", ctypes.c_int64), ("Q", ctypes.c_void_p), ("ldq", ctypes.c_int64),
                ("R", ctypes.c_void_p), ("ldr", ctypes.c_int64), ("work", ctypes.c_void_p)]


class mgsa_group_member(ctypes.Structure):
    _fields_ = [("job", mgsa_job), ("first", ctypes.c_int32), ("count", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


MGSA_GROUP_MAX = 64
MGSA_BATCH_MAX_N = 256
MGSA_BATCH_INFO_INVALID = -2147483647


class MgsaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_lock = threading.Lock()

# Every exported entry point and its ctypes signature (kept in step with include/mgsa.h).
_VP, _I64, _INT, _SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
SIGNATURES = {
    "mgsa_create": (_INT, [ctypes.POINTER(_VP), _INT]),
    "mgsa_destroy": (_INT, [_VP]),
    "mgsa_reserve": (_INT, [_VP, _I64, _INT, _INT]),
    "mgsa_workspace_bytes": (_SZ, [_VP, _I64, _INT, _INT]),
    "mgsa_qr": (_INT, [_VP, ctypes.POINTER(mgsa_csr), _VP, _I64, _INT, _I64, _INT, _VP, _I64, _VP, _INT, _VP]),
    "mgsa_qr_steps": (_INT, [_VP, ctypes.POINTER(mgsa_csr), _VP, _I64, _INT, _I64, _INT, _VP, _I64, _VP, _INT, _INT,
                             _INT, _VP]),
    "mgsa_get_info": (_INT, [_VP, _VP, ctypes.POINTER(_INT)]),
    "mgsa_copy_info": (_INT, [_VP, _VP, _VP]),
    "mgsa_qr_host": (_INT, [_VP, _VP, _VP, _VP, _I64, _VP, _I64, _INT, _I64, _INT, _VP, _I64, _VP, _INT, _VP,
                            ctypes.POINTER(_INT)]),
    "mgsa_set_param": (_INT, [_VP, _INT, _I64]),
    "mgsa_qr_noalloc": (_INT, [ctypes.POINTER(mgsa_csr), _VP, _I64, _INT, _I64, _INT, _VP, _I64, _VP, _INT, _VP, _VP]),
    "mgsa_job_workspace_bytes": (_SZ, [_I64, _INT, _INT]),
    "mgsa_qr_batched": (_INT, [_VP, _INT, _VP, _VP, _VP]),
    "mgsa_qr_append": (_INT, [_VP, ctypes.POINTER(mgsa_csr), _VP, _I64, _VP, _I64, _INT, _VP, _I64, _INT, _I64, _INT,
                              _VP, _I64, _VP, _I64, _VP, _INT, _VP]),
    "mgsa_group_workspace_bytes": (_SZ, [_VP, _I64, _INT, _INT]),
    "mgsa_qr_group": (_INT, [_VP, _INT, _INT, ctypes.POINTER(mgsa_group_member), _VP]),
    "mgsa_fp64_probe": (_INT, [_INT, _INT, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "mgsa_last_error": (ctypes.c_char_p, []),
}
(MGSA_PARAM_MAX_CTAS, MGSA_PARAM_CHUNK_ROWS, MGSA_PARAM_MIN_ROWS_PER_CTA, MGSA_PARAM_BATCH_CTAS, MGSA_PARAM_ROW_MODE,
 MGSA_PARAM_SPMM_PANEL, MGSA_PARAM_CLUSTER, MGSA_PARAM_WAIT_FAULT) = 0, 1, 2, 3, 4, 5, 6, 7


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libmgsa (built in-tree on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB if os.path.exists(_build.LIB) else _build.build()
            handle = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("device tensor expected")
        return x.data_ptr()
    return int(x)


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def _check(status: int):
    if status != MGSA_OK:
        raise MgsaError(status, lib().mgsa_last_error().decode())


def mgsa_last_error() -> str:
    return lib().mgsa_last_error().decode()


def mgsa_fp64_probe(device: int = 0, iters: int = 20000) -> tuple[float, float]:
    """Measured FP64 FMA rate of the device: ``(TFLOP/s, ms of the timed launch)``."""
    tf, ms = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().mgsa_fp64_probe(device, iters, ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def mgsa_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().mgsa_create(ctypes.byref(h), device))
    return h.value


def mgsa_destroy(h: int) -> None:
    _check(lib().mgsa_destroy(h))


def mgsa_reserve(h: int, m: int, n: int, variant: int) -> None:
    _check(lib().mgsa_reserve(h, m, n, variant))


def mgsa_workspace_bytes(h: int, m: int, n: int, variant: int) -> int:
    return int(lib().mgsa_workspace_bytes(h, m, n, variant))


def mgsa_set_param(h: int, param: int, value: int) -> None:
    _check(lib().mgsa_set_param(h, param, value))


def make_csr(m: int, nnz: int, rowptr, col, val) -> mgsa_csr:
    return mgsa_csr(m, nnz, _ptr(rowptr), _ptr(col), _ptr(val))


def mgsa_qr(h: int, A: mgsa_csr, Z, m: int, n: int, ldz: int, variant: int, Q, ldq: int, R, ldr: int,
            stream=None) -> int:
    """Queue one QR; returns the status (MGSA_OK or an argument error)."""
    return int(lib().mgsa_qr(h, ctypes.byref(A), _ptr(Z), m, n, ldz, variant, _ptr(Q), ldq, _ptr(R), ldr,
                             _stream(stream)))


def mgsa_qr_append(h: int, A: mgsa_csr, Qold, ldqo: int, Pold, ldpo: int, k: int, Z, m: int, n: int, ldz: int,
                   variant: int, Q, ldq: int, P, ldp: int, R, ldr: int, stream=None) -> int:
    """Queue the orthogonalisation of Z against k given columns (Qold, Pold);
    returns the status of the call.  ``P`` may be None."""
    return int(lib().mgsa_qr_append(h, ctypes.byref(A), _ptr(Qold), ldqo, _ptr(Pold), ldpo, k, _ptr(Z), m, n, ldz,
                                    variant, _ptr(Q), ldq, _ptr(P), ldp, _ptr(R), ldr, _stream(stream)))


def mgsa_qr_steps(h: int, A: mgsa_csr, Z, m: int, n: int, ldz: int, variant: int, Q, ldq: int, R, ldr: int,
                  first: int, count: int, stream=None) -> int:
    """Queue steps [first, first + count) of a time-sliced QR; returns the status of the call."""
    return int(lib().mgsa_qr_steps(h, ctypes.byref(A), _ptr(Z), m, n, ldz, variant, _ptr(Q), ldq, _ptr(R), ldr, first,
                                   count, _stream(stream)))


def mgsa_qr_noalloc(A: mgsa_csr, Z, m: int, n: int, ldz: int, variant: int, Q, ldq: int, R, ldr: int, info_dev=None,
                    stream=None) -> int:
    """Queue one QR whose scratch is the library's static device array (no
    allocation, no handle); returns the status of the call."""
    return int(lib().mgsa_qr_noalloc(ctypes.byref(A), _ptr(Z), m, n, ldz, variant, _ptr(Q), ldq, _ptr(R), ldr,
                                     _ptr(info_dev), _stream(stream)))


def mgsa_job_workspace_bytes(m: int, n: int, variant: int) -> int:
    return int(lib().mgsa_job_workspace_bytes(m, n, variant))


def mgsa_qr_batched(h: int, count: int, jobs_dev, info_dev, stream=None) -> int:
    """Queue a batch; ``jobs_dev`` is a device buffer holding ``count``
    ``mgsa_job`` structs, ``info_dev`` a device int32 buffer of ``count``."""
    return int(lib().mgsa_qr_batched(h, count, _ptr(jobs_dev), _ptr(info_dev), _stream(stream)))


def mgsa_group_workspace_bytes(h: int, m: int, n: int, variant: int) -> int:
    return int(lib().mgsa_group_workspace_bytes(h, m, n, variant))


def mgsa_qr_group(h: int, variant: int, members, stream=None) -> int:
    """Queue one grouped launch; ``members`` is a sequence of
    ``mgsa_group_member``; returns the status of the call."""
    arr = (mgsa_group_member * len(members))(*members)
    return int(lib().mgsa_qr_group(h, variant, len(members), arr, _stream(stream)))


def group_member(m: int, n: int, variant: int, rowptr, col, val, Z, ldz: int, Q, ldq: int, R, ldr: int, work,
                 first: int, count: int, ctas: int) -> mgsa_group_member:
    job = mgsa_job(m, n, variant, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(Z), ldz, _ptr(Q), ldq, _ptr(R), ldr,
                   _ptr(work))
    return mgsa_group_member(job, first, count, ctas, 0)


def mgsa_copy_info(h: int, info_dev, stream=None) -> None:
    _check(lib().mgsa_copy_info(h, _ptr(info_dev), _stream(stream)))


def mgsa_get_info(h: int, stream=None) -> tuple[int, int]:
    info = ctypes.c_int(0)
    st = lib().mgsa_get_info(h, _stream(stream), ctypes.byref(info))
    return int(st), int(info.value)


def mgsa_qr_host(h: int, rowptr, col, val, nnz: int, Z, m: int, n: int, ldz: int, variant: int, Q, ldq: int, R,
                 ldr: int, stream=None) -> tuple[int, int]:
    """Host-buffer QR (numpy arrays or pinned torch CPU tensors); returns (status, info)."""
    def hp(a):
        if hasattr(a, "ctypes"):
            return a.ctypes.data
        return a.data_ptr()
    info = ctypes.c_int(0)
    st = lib().mgsa_qr_host(h, hp(rowptr), hp(col), hp(val), nnz, hp(Z), m, n, ldz, variant, hp(Q), ldq, hp(R), ldr,
                            _stream(stream), ctypes.byref(info))
    return int(st), int(info.value)


# ---------------------------------------------------------------------------
# Convenience layer on torch tensors (allocation of Q/R + marshalling).
# ---------------------------------------------------------------------------

class Handle:
    """Owns one mgsa handle; ``qr`` runs a QR on device tensors."""

    def __init__(self, device: int = 0):
        self.device = device
        self.h = mgsa_create(device)

    def close(self):
        if self.h:
            mgsa_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def qr_into(self, A, Z, Q, R, variant, stream=None) -> None:
        """``A`` = (rowptr, col, val) CUDA tensors; ``Z``/``Q`` (m, n) and ``R``
        (n, n) column-major CUDA float64 views (``t.T`` of a row-major (n, m))."""
        rowptr, col, val = A
        m, n = Z.shape
        for t in (Z, Q, R):
            if t.dtype.itemsize != 8 or t.stride(0) != 1:
                raise ValueError("Z, Q, R must be column-major float64 (stride(0) == 1)")
        v = VARIANTS[variant] if isinstance(variant, str) else variant
        csr = make_csr(m, col.numel(), rowptr, col, val)
        st = mgsa_qr(self.h, csr, Z, m, n, Z.stride(1), v, Q, Q.stride(1), R, R.stride(1), stream)
        _check(st)

    def qr(self, A, Z, variant, stream=None):
        """Allocate column-major Q, R and queue the QR; returns (Q, R)."""
        import torch
        m, n = Z.shape
        Q = torch.empty((n, m), dtype=torch.float64, device=Z.device).T
        R = torch.empty((n, n), dtype=torch.float64, device=Z.device).T
        self.qr_into(A, Z, Q, R, variant, stream)
        return Q, R

    def append(self, A, Qold, Pold, Z, variant, want_p: bool = True, stream=None):
        """Orthonormalise the columns of ``Z`` against the given A-orthonormal
        ``Qold`` (with ``Pold`` = its p_i; both None for none) and among
        themselves.  Returns column-major ``(Q, P, R)``, R of shape (k+n, n);
        P is None unless ``want_p``."""
        import torch
        rowptr, col, val = A
        m, n = Z.shape
        k = 0 if Qold is None else Qold.shape[1]
        dev = Z.device
        Q = torch.empty((n, m), dtype=torch.float64, device=dev).T
        P = torch.empty((n, m), dtype=torch.float64, device=dev).T if want_p else None
        R = torch.empty((n, k + n), dtype=torch.float64, device=dev).T
        for t in [Z, Q, R] + ([P] if want_p else []) + ([Qold, Pold] if k else []):
            if t.dtype.itemsize != 8 or t.stride(0) != 1:
                raise ValueError("all matrices must be column-major float64 (stride(0) == 1)")
        v = VARIANTS[variant] if isinstance(variant, str) else variant
        csr = make_csr(m, col.numel(), rowptr, col, val)
        st = mgsa_qr_append(self.h, csr, Qold, Qold.stride(1) if k else m, Pold, Pold.stride(1) if k else m, k, Z, m,
                            n, Z.stride(1), v, Q, Q.stride(1), P, P.stride(1) if want_p else m, R, R.stride(1),
                            stream)
        _check(st)
        return Q, P, R

    def set_param(self, param: int, value: int) -> None:
        mgsa_set_param(self.h, param, value)

    def info(self, stream=None) -> tuple[int, int]:
        return mgsa_get_info(self.h, stream)
