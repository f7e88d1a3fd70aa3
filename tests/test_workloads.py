"""The seeded generators produce the structures the workloads name."""
import numpy as np
import pytest

import workloads as W


def _sym_check(A):
    D = W.csr_to_dense(A)
    assert np.array_equal(D, D.T)
    rowptr, col, _ = A
    for i in range(len(rowptr) - 1):
        c = col[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    return D


def test_tridiag():
    A = W.tridiag_csr(50)
    D = _sym_check(A)
    assert len(A[1]) == 3 * 50 - 2
    assert np.all(np.diag(D) == 2.1)


def test_laplace2d_nnz_and_values():
    side = 16
    A = W.laplace2d_csr(side, side, 0.01)
    D = _sym_check(A)
    assert len(A[1]) == 5 * side * side - 4 * side
    assert np.allclose(np.diag(D), 4.01)
    assert np.linalg.eigvalsh(D).min() > 0.01


def test_poisson2d_full_size_nnz():
    A = W.laplace2d_csr(512, 512, 0.01)
    assert len(A[1]) == 1308672


@pytest.mark.parametrize("side", [5, 9])
def test_varcoef3d_structure(side):
    A = W.varcoef3d_csr(side)
    D = _sym_check(A)
    assert len(A[1]) == 7 * side ** 3 - 6 * side ** 2
    off = D - np.diag(np.diag(D))
    assert np.all(off <= 0)
    # diagonal = sum of face coefficients + shift >= |off-diagonal row sum| + shift
    assert np.all(np.diag(D) - np.abs(off).sum(axis=1) >= 1e-3 - 1e-12)
    assert np.linalg.eigvalsh(D).min() > 0


def test_banded_spd():
    A = W.banded_spd_csr(40, 8, W.rng(1, 2))
    D = _sym_check(A)
    off = D - np.diag(np.diag(D))
    assert np.allclose(np.diag(D), 1.0 + np.abs(off).sum(axis=1))
    assert np.abs(np.triu(off, 9)).max() == 0.0
    assert np.linalg.eigvalsh(D).min() > 0.0


def test_graded_Z_condition():
    Z = W.graded_Z(4000, 64)
    assert Z.flags.f_contiguous
    s = np.linalg.svd(Z, compute_uv=False)
    assert 3e5 < s[0] / s[-1] < 3e6


def test_generators_are_deterministic():
    a1, z1 = W.banded(300, 10, seed=3, index=7)
    a2, z2 = W.banded(300, 10, seed=3, index=7)
    assert all(np.array_equal(x, y) for x, y in zip(a1, a2)) and np.array_equal(z1, z2)


def test_batch_sizes_ranges():
    ms, ns = W.batch_sizes(4096)
    assert ms.min() >= 256 and ms.max() <= 8192
    assert ns.min() == 4 and ns.max() == 64
    assert np.all(ms >= ns)


def test_exp2_problem_conditions():
    A, Z, dsel = W.exp2_problem(6.0, 4.0, case=2)
    ev = np.linalg.eigvalsh(A)
    assert abs(np.log10(ev.max() / ev.min()) - 6.0) < 1e-6
    L = np.linalg.cholesky(A)
    s = np.linalg.svd(L.T @ Z, compute_uv=False)
    assert abs(np.log10(s[0] / s[-1]) - 4.0) < 1e-6
