"""CPU oracle for the A-inner-product MGS thin QR (arXiv 1703.10440).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package.  It shares no code with the CUDA library; the only module both sides
use is ``workloads`` (seeded input generators, no arithmetic of the method).

Everything here is a thin ctypes wrapper around ``mgs_oracle.c``:

* :func:`mgs` runs one of Algorithms 3-8 of the paper (naive / HA / HP, column-
  or row-oriented) in plain FP64 C and returns ``(Q, R, info, kind, mv_count)``.
* :func:`cgs` runs the classical Gram-Schmidt counterparts (CGS-naive / HA /
  HP, both forms), :func:`mgs_append` continues the column form after k given
  A-orthonormal columns.
* :func:`mgs_par` runs the row-oriented Algorithms 4 / 7 / 8 on several host
  cores (``mgs_oracle_par.c``); it performs the same operations in the same
  order as :func:`mgs` and returns the same bits.
* :func:`repr_error`, :func:`orth_loss` and :func:`chol_gram` evaluate the
  representation error ``||Z - QR||_F / ||Z||_F``, the loss of A-orthogonality
  ``||I - Q^T A Q||_F`` (both in double-double) and the long-double Cholesky
  factor of ``Z^T A Z``.

Parity status of each function is recorded next to it; every function here is
pinned by tests under ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

VARIANTS = {"naive": 0, "ha": 1, "hp": 2}
FORMS = {"col": 0, "row": 1}

_lib = None


def load(path: str | None = None):
    """Load (building if needed) the oracle shared library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(_build.build()))
    return _lib


def _bind(lib):
    i64, i32, dp, ip = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p
    lib.oracle_mgs.restype = ctypes.c_int
    lib.oracle_mgs.argtypes = [i32, i32, i64, i32, ip, ip, dp, dp, i64, dp, i64, dp, i32,
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]
    lib.oracle_cgs.restype = ctypes.c_int
    lib.oracle_cgs.argtypes = lib.oracle_mgs.argtypes
    lib.oracle_mgs_append.restype = ctypes.c_int
    lib.oracle_mgs_append.argtypes = [i32, i64, i32, i32, ip, ip, dp, dp, i64, dp, i64, dp, i64, dp, i64, dp, i64, dp,
                                      i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]
    lib.oracle_csr_mv.restype = None
    lib.oracle_csr_mv.argtypes = [i64, ip, ip, dp, dp, dp]
    lib.oracle_repr_error.restype = None
    lib.oracle_repr_error.argtypes = [i64, i32, dp, i64, dp, i64, dp, i32,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.oracle_orth_loss.restype = ctypes.c_double
    lib.oracle_orth_loss.argtypes = [i64, i32, ip, ip, dp, dp, i64, dp]
    lib.oracle_chol_gram_ld.restype = ctypes.c_int
    lib.oracle_chol_gram_ld.argtypes = [i64, i32, ip, ip, dp, dp, i64, dp, i32]
    return lib


_par_lib = None


def load_par():
    """Load (building if needed) the multi-core build of the row-oriented
    algorithms (``mgs_oracle_par.c``)."""
    global _par_lib
    if _par_lib is None:
        lib = ctypes.CDLL(_build.build_par())
        i64, i32, p = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_par_mgs_row.restype = ctypes.c_int
        lib.oracle_par_mgs_row.argtypes = [i32, i64, i32, p, p, p, p, i64, p, i64, p, i32, ctypes.POINTER(ctypes.c_int)]
        lib.oracle_par_threads.restype = ctypes.c_int
        lib.oracle_par_threads.argtypes = []
        lib.oracle_par_set_threads.restype = None
        lib.oracle_par_set_threads.argtypes = [i32]
        _par_lib = lib
    return _par_lib


def par_threads(threads: int | None = None) -> int:
    """Set (if given) and return the thread count of :func:`mgs_par`."""
    lib = load_par()
    if threads:
        lib.oracle_par_set_threads(int(threads))
    return int(lib.oracle_par_threads())


def mgs_par(A, Z: np.ndarray, variant: str = "naive", threads: int | None = None):
    """Algorithm 4 / 7 / 8 (row form) on several host cores: the same
    operations as ``mgs(A, Z, variant, "row")`` in the same order, so the same
    bits, with independent rows and columns spread over OpenMP threads.
    Returns ``(Q, R, info, kind)``.  Parity: pinned bitwise to :func:`mgs` by
    ``tests/test_oracle_par.py``."""
    lib = load_par()
    if threads:
        lib.oracle_par_set_threads(int(threads))
    rowptr, col, val = _csr_arrays(A)
    Zf = _fortran(Z)
    m, n = Zf.shape
    Q = np.empty((m, n), dtype=np.float64, order="F")
    R = np.empty((n, n), dtype=np.float64, order="F")
    kind = ctypes.c_int(0)
    info = lib.oracle_par_mgs_row(VARIANTS[variant], m, n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(Zf), m, _ptr(Q),
                                  m, _ptr(R), n, ctypes.byref(kind))
    if info < 0:
        raise ValueError("oracle_par_mgs_row: invalid arguments")
    return Q, R, int(info), int(kind.value)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr_arrays(A):
    rowptr = np.ascontiguousarray(A[0], dtype=np.int32)
    col = np.ascontiguousarray(A[1], dtype=np.int32)
    val = np.ascontiguousarray(A[2], dtype=np.float64)
    return rowptr, col, val


def _fortran(Z: np.ndarray) -> np.ndarray:
    return np.asfortranarray(Z, dtype=np.float64)


def mgs(A, Z: np.ndarray, variant: str = "naive", form: str = "col", lib=None):
    """Run Algorithm 3/4 (naive), 5/7 (HA) or 6/8 (HP) on the CPU.

    ``A`` is ``(rowptr, col, val)`` (CSR, int32/int32/float64); ``Z`` is an
    ``m x n`` float64 array.  Returns ``(Q, R, info, kind, mv_count)`` where
    ``info`` is 0 or the 1-based breakdown column, ``kind`` 1 = non-positive
    ``z^T x``, 2 = NaN/Inf, and ``mv_count`` counts sparse matrix-vector
    products (the HP block product ``AZ`` counts once).
    """
    lib = lib or load()
    rowptr, col, val = _csr_arrays(A)
    Zf = _fortran(Z)
    m, n = Zf.shape
    Q = np.zeros((m, n), dtype=np.float64, order="F")
    R = np.zeros((n, n), dtype=np.float64, order="F")
    mv = ctypes.c_int64(0)
    kind = ctypes.c_int(0)
    info = lib.oracle_mgs(VARIANTS[variant], FORMS[form], m, n, _ptr(rowptr), _ptr(col), _ptr(val),
                          _ptr(Zf), m, _ptr(Q), m, _ptr(R), n, ctypes.byref(mv), ctypes.byref(kind))
    if info < 0:
        raise ValueError("oracle_mgs: invalid arguments")
    return Q, R, int(info), int(kind.value), int(mv.value)


def cgs(A, Z: np.ndarray, variant: str = "naive", form: str = "col", lib=None):
    """Classical Gram-Schmidt counterpart of :func:`mgs` (Sections 2.3 and
    3.3): the same algorithms with r_ij = p_i^T z_j^{(0)}.  Same arguments and
    return value as :func:`mgs`."""
    lib = lib or load()
    rowptr, col, val = _csr_arrays(A)
    Zf = _fortran(Z)
    m, n = Zf.shape
    Q = np.zeros((m, n), dtype=np.float64, order="F")
    R = np.zeros((n, n), dtype=np.float64, order="F")
    mv = ctypes.c_int64(0)
    kind = ctypes.c_int(0)
    info = lib.oracle_cgs(VARIANTS[variant], FORMS[form], m, n, _ptr(rowptr), _ptr(col), _ptr(val),
                          _ptr(Zf), m, _ptr(Q), m, _ptr(R), n, ctypes.byref(mv), ctypes.byref(kind))
    if info < 0:
        raise ValueError("oracle_cgs: invalid arguments")
    return Q, R, int(info), int(kind.value), int(mv.value)


def mgs_append(A, Qo, Po, Z: np.ndarray, variant: str = "naive", lib=None):
    """Successive orthogonalisation: continue Algorithm 3/5/6 (column form)
    with k given columns ``Qo`` (A-orthonormal) and ``Po`` (their p_i), then
    the n columns of ``Z``.  Returns ``(Q, P, R, info, kind, mv_count)`` with
    R of shape (k+n, n).  ``Qo = Po = None`` (k = 0) is Algorithm 3/5/6."""
    lib = lib or load()
    rowptr, col, val = _csr_arrays(A)
    Zf = _fortran(Z)
    m, n = Zf.shape
    if Qo is None:
        k, Qof, Pof = 0, np.zeros((m, 1), order="F"), np.zeros((m, 1), order="F")
    else:
        Qof, Pof = _fortran(Qo), _fortran(Po)
        k = Qof.shape[1]
    Q = np.zeros((m, n), dtype=np.float64, order="F")
    P = np.zeros((m, n), dtype=np.float64, order="F")
    R = np.zeros((k + n, n), dtype=np.float64, order="F")
    mv = ctypes.c_int64(0)
    kind = ctypes.c_int(0)
    info = lib.oracle_mgs_append(VARIANTS[variant], m, k, n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(Qof), m,
                                 _ptr(Pof), m, _ptr(Zf), m, _ptr(Q), m, _ptr(P), m, _ptr(R), k + n,
                                 ctypes.byref(mv), ctypes.byref(kind))
    if info < 0:
        raise ValueError("oracle_mgs_append: invalid arguments")
    return Q, P, R, int(info), int(kind.value), int(mv.value)


def csr_mv(A, x: np.ndarray, lib=None) -> np.ndarray:
    lib = lib or load()
    rowptr, col, val = _csr_arrays(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib.oracle_csr_mv(len(rowptr) - 1, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
    return y


def repr_error(Z: np.ndarray, Q: np.ndarray, R: np.ndarray, lib=None) -> float:
    """``||Z - QR||_F / ||Z||_F`` with every entry of ``Z - QR`` in double-double."""
    lib = lib or load()
    Zf, Qf, Rf = _fortran(Z), _fortran(Q), _fortran(R)
    m, n = Zf.shape
    e, z = ctypes.c_double(0), ctypes.c_double(0)
    lib.oracle_repr_error(m, n, _ptr(Zf), m, _ptr(Qf), m, _ptr(Rf), n, ctypes.byref(e), ctypes.byref(z))
    return e.value / z.value


def orth_loss(A, Q: np.ndarray, lib=None, return_gram: bool = False):
    """``||I - Q^T A Q||_F`` with ``A Q`` and the Gram matrix in double-double."""
    lib = lib or load()
    rowptr, col, val = _csr_arrays(A)
    Qf = _fortran(Q)
    m, n = Qf.shape
    G = np.zeros((n, n), dtype=np.float64, order="F")
    loss = lib.oracle_orth_loss(m, n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(Qf), m, _ptr(G))
    return (loss, G) if return_gram else loss


def chol_gram(A, Z: np.ndarray, lib=None):
    """Upper Cholesky factor of ``Z^T A Z`` in long double; returns ``(R, info)``."""
    lib = lib or load()
    rowptr, col, val = _csr_arrays(A)
    Zf = _fortran(Z)
    m, n = Zf.shape
    R = np.zeros((n, n), dtype=np.float64, order="F")
    info = lib.oracle_chol_gram_ld(m, n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(Zf), m, _ptr(R), n)
    return R, int(info)
