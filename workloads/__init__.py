"""Seeded synthetic inputs for the A-inner-product MGS thin QR.

This module is the only code that both the CUDA path (through its tests and
``bench.py``) and the CPU oracle use.  It draws matrices; it performs none of
the method's arithmetic.  Every array comes from its own PCG64 stream
``Generator(PCG64(SeedSequence([seed, tag])))`` so that any single array can be
regenerated on its own.

Sparse matrices are returned as ``(rowptr, col, val)`` numpy arrays (int32,
int32, float64), both triangles stored, columns ascending within each row.
Dense ``Z`` matrices are returned Fortran-ordered (column-major) float64.

Workloads (the paper's own matrices, a dense random SPD matrix and the
AUNW9180 overlap matrix of Section 4.1, are not available; these synthetic
families stand in for them):

* ``tridiag``        tridiag(-1, 2.1, -1), m = 4096, Z = N(0,1) m x 16;
* ``poisson2d``      5-point Laplacian on a 512 x 512 grid + 0.01 I,
                     Z = G diag(logspace(0, -6, 64)), kappa(Z) ~ 1e6;
* ``varcoef3d``      7-point variable-coefficient Laplacian on 128^3 with cell
                     coefficients exp(N(0,1)), face coefficient = mean of the
                     two cells, Dirichlet boundary, + 1e-3 I; Z = N(0,1) x 128;
* ``banded``         random banded SPD, half-bandwidth 8, off-diagonals
                     U(-1, 1) mirrored, diagonal 1 + row |off-diagonal| sum;
* ``batch``          4096 banded instances with m ~ logU[256, 8192],
                     n ~ U{4..64};
* ``exp2``           Section 4.2's A = V D V^T, Z = U E W^T test family;
* ``denseband``      banded SPD with half-bandwidth 194 and m = 9180: about
                     389 nonzeros per row and 3.5e6 in all, the size and
                     density of the sparse matrix of Section 4.1, Z = N(0,1).
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20170330

# Stream tags, one per array role.
TAG_Z = 1
TAG_COEF = 2
TAG_BAND = 3
TAG_SIZES = 4
TAG_V = 5
TAG_W = 6


def rng(seed: int, tag: int, *extra: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, tag, *extra])))


# --------------------------------------------------------------------------
# CSR assembly from per-row stencils
# --------------------------------------------------------------------------

def _stencil_to_csr(cols: np.ndarray, vals: np.ndarray, mask: np.ndarray):
    """``cols``/``vals``/``mask`` are (m, s) arrays whose columns are ordered by
    ascending column index within each row; masked-out entries are dropped."""
    m = cols.shape[0]
    counts = mask.sum(axis=1).astype(np.int64)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    col = cols[mask].astype(np.int32)
    val = vals[mask].astype(np.float64)
    return rowptr.astype(np.int32), col, val


def tridiag_csr(m: int, diag: float = 2.1, off: float = -1.0):
    k = np.arange(m, dtype=np.int64)
    cols = np.stack([k - 1, k, k + 1], axis=1)
    vals = np.stack([np.full(m, off), np.full(m, diag), np.full(m, off)], axis=1)
    mask = (cols >= 0) & (cols < m)
    return _stencil_to_csr(cols, vals, mask)


def laplace2d_csr(nx: int, ny: int, shift: float):
    """5-point Laplacian (diag 4 + shift, neighbours -1, no h^2 scaling,
    Dirichlet boundary) on an nx x ny grid, row index k = ix + nx*iy."""
    m = nx * ny
    k = np.arange(m, dtype=np.int64)
    ix, iy = k % nx, k // nx
    cols = np.stack([k - nx, k - 1, k, k + 1, k + nx], axis=1)
    ones = np.ones(m)
    vals = np.stack([-ones, -ones, (4.0 + shift) * ones, -ones, -ones], axis=1)
    mask = np.stack([iy > 0, ix > 0, np.ones(m, bool), ix < nx - 1, iy < ny - 1], axis=1)
    return _stencil_to_csr(cols, vals, mask)


def varcoef3d_csr(n1: int, seed: int = SEED, shift: float = 1e-3):
    """7-point variable-coefficient Laplacian on an n1^3 grid.

    Cell coefficients c_k = exp(N(0,1)); the face between cells k and l has
    coefficient (c_k + c_l)/2 and contributes -face to A[k,l]; a boundary face
    of cell k contributes c_k to the diagonal only (Dirichlet).  Diagonal =
    sum of the six face coefficients + shift."""
    nx = ny = nz = n1
    m = nx * ny * nz
    c = np.exp(rng(seed, TAG_COEF).standard_normal(m))
    k = np.arange(m, dtype=np.int64)
    ix, iy, iz = k % nx, (k // nx) % ny, k // (nx * ny)
    offs = [(-nx * ny, iz > 0), (-nx, iy > 0), (-1, ix > 0), (1, ix < nx - 1), (nx, iy < ny - 1), (nx * ny, iz < nz - 1)]
    diag = np.full(m, shift)
    cols_l, vals_l, mask_l = [], [], []
    for off, inside in offs:
        nb = np.where(inside, k + off, k)
        face = np.where(inside, 0.5 * (c + c[nb]), c)
        diag += face
        cols_l.append(k + off)
        vals_l.append(-face)
        mask_l.append(inside)
    # order by ascending column: -nxny, -nx, -1, 0, +1, +nx, +nxny
    cols = np.stack(cols_l[:3] + [k] + cols_l[3:], axis=1)
    vals = np.stack(vals_l[:3] + [diag] + vals_l[3:], axis=1)
    mask = np.stack(mask_l[:3] + [np.ones(m, bool)] + mask_l[3:], axis=1)
    return _stencil_to_csr(cols, vals, mask)


def banded_spd_csr(m: int, hb: int, gen: np.random.Generator):
    """Symmetric banded matrix: upper band U(-1,1) mirrored; diagonal
    1 + sum of |off-diagonals| of the row (strictly diagonally dominant)."""
    k = np.arange(m, dtype=np.int64)
    up = gen.uniform(-1.0, 1.0, size=(m, hb))  # up[k, d-1] = A[k, k+d]
    upmask = (k[:, None] + np.arange(1, hb + 1)[None, :]) < m
    up = np.where(upmask, up, 0.0)
    lo = np.zeros((m, hb))  # lo[k, d-1] = A[k, k-d] = up[k-d, d-1]
    for d in range(1, min(hb, m - 1) + 1):
        lo[d:, d - 1] = up[: m - d, d - 1]
    lomask = (k[:, None] - np.arange(1, hb + 1)[None, :]) >= 0
    diag = 1.0 + np.abs(up).sum(axis=1) + np.abs(lo).sum(axis=1)
    # ascending columns: k-hb .. k-1, k, k+1 .. k+hb
    cols = np.concatenate([k[:, None] - np.arange(hb, 0, -1)[None, :], k[:, None],
                           k[:, None] + np.arange(1, hb + 1)[None, :]], axis=1)
    vals = np.concatenate([lo[:, ::-1], diag[:, None], up], axis=1)
    mask = np.concatenate([lomask[:, ::-1], np.ones((m, 1), bool), upmask], axis=1)
    return _stencil_to_csr(cols, vals, mask)


def dense_csr(A: np.ndarray):
    """Dense matrix stored as CSR with full rows (test-sized problems)."""
    m = A.shape[0]
    cols = np.tile(np.arange(m, dtype=np.int64), (m, 1))
    return _stencil_to_csr(cols, np.asarray(A, dtype=np.float64), np.ones((m, m), bool))


def csr_to_dense(A) -> np.ndarray:
    rowptr, col, val = A
    m = len(rowptr) - 1
    D = np.zeros((m, m))
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    np.add.at(D, (rows, col), val)
    return D


# --------------------------------------------------------------------------
# Z matrices
# --------------------------------------------------------------------------

def gaussian_Z(m: int, n: int, seed: int = SEED, tag: int = TAG_Z, *extra: int) -> np.ndarray:
    """iid N(0,1), column-major: column j is the j-th block of m draws."""
    return rng(seed, tag, *extra).standard_normal((n, m)).T


def graded_Z(m: int, n: int, seed: int = SEED, lo_exp: float = -6.0) -> np.ndarray:
    """G diag(logspace(0, lo_exp, n)) with G iid N(0,1)."""
    G = gaussian_Z(m, n, seed)
    d = np.logspace(0.0, lo_exp, n)
    return G * d[None, :]


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

def tridiag(m: int = 4096, n: int = 16, seed: int = SEED):
    return tridiag_csr(m), gaussian_Z(m, n, seed)


def poisson2d(side: int = 512, n: int = 64, seed: int = SEED, shift: float = 0.01, lo_exp: float = -6.0):
    return laplace2d_csr(side, side, shift), graded_Z(side * side, n, seed, lo_exp)


def varcoef3d(side: int = 128, n: int = 128, seed: int = SEED, shift: float = 1e-3):
    return varcoef3d_csr(side, seed, shift), gaussian_Z(side ** 3, n, seed)


def banded(m: int, n: int, seed: int = SEED, hb: int = 8, index: int = 0):
    A = banded_spd_csr(m, hb, rng(seed, TAG_BAND, index))
    return A, gaussian_Z(m, n, seed, TAG_Z, index)


def denseband(m: int = 9180, n: int = 50, hb: int = 194, seed: int = SEED):
    """Dense-band SPD matrix (long CSR rows) and Gaussian Z."""
    A = banded_spd_csr(m, hb, rng(seed, TAG_BAND, 194))
    return A, gaussian_Z(m, n, seed, TAG_Z, 194)


def batch_sizes(count: int = 4096, seed: int = SEED, m_lo: int = 256, m_hi: int = 8192, n_lo: int = 4, n_hi: int = 64):
    """(m, n) per instance: m = round(exp(U(ln m_lo, ln m_hi))), n ~ U{n_lo..n_hi}, m >= n."""
    g = rng(seed, TAG_SIZES)
    ms = np.rint(np.exp(g.uniform(math.log(m_lo), math.log(m_hi), size=count))).astype(np.int64)
    ns = g.integers(n_lo, n_hi + 1, size=count).astype(np.int64)
    ms = np.maximum(ms, ns)
    return ms, ns


def batch(count: int = 4096, seed: int = SEED, **kw):
    """List of (A, Z) banded instances with the sizes of :func:`batch_sizes`."""
    ms, ns = batch_sizes(count, seed, **kw)
    return [banded(int(m), int(n), seed, 8, i) for i, (m, n) in enumerate(zip(ms, ns))]


# --------------------------------------------------------------------------
# Section 4.2 accuracy family (A = V D V^T, Z = U E W^T)
# --------------------------------------------------------------------------

def random_orthogonal(k: int, gen: np.random.Generator) -> np.ndarray:
    Gm = gen.standard_normal((k, k))
    Qm, Rm = np.linalg.qr(Gm)
    return Qm * np.sign(np.diag(Rm))[None, :]


def exp2_problem(log_kA: float, log_kAZ: float, case: int, m: int = 100, n: int = 20, seed: int = SEED, index: int = 0):
    """A = V D V^T with log10 d_i evenly spaced over [0, log_kA]; Z = U E W^T
    with U the eigenvectors of the n largest (case 1) or n smallest (case 2)
    eigenvalues.  E is chosen so that the singular values of A^{1/2} Z are
    evenly spaced in log scale over [0, log_kAZ] (kappa(A^{1/2} Z) = 10^log_kAZ).
    Returns (A_dense, Z, d_selected)."""
    V = random_orthogonal(m, rng(seed, TAG_V, index))
    W = random_orthogonal(n, rng(seed, TAG_W, index))
    alpha = log_kA / (m - 1)
    d = 10.0 ** (alpha * np.arange(m))
    A = (V * d[None, :]) @ V.T
    A = 0.5 * (A + A.T)
    sel = np.arange(m - n, m) if case == 1 else np.arange(n)
    U = V[:, sel]
    sv = 10.0 ** (log_kAZ / (n - 1) * np.arange(n)) if n > 1 else np.ones(1)
    e = sv / np.sqrt(d[sel])
    Z = (U * e[None, :]) @ W.T
    return A, np.asfortranarray(Z), d[sel]
