"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each pin checks the oracle against something other than itself:

* A = I reduces MGS to the textbook QR: R and Q equal Householder QR
  (numpy.linalg.qr) with the signs fixed so that diag(R) > 0.
* Cholesky reduction (Section 1, eq. (1)): R is the upper Cholesky factor of
  Z^T A Z, computed here in 50-digit mpmath from the exact binary inputs.
* Closed form: tridiag(-1, 2.1, -1) has the sine eigenvectors, so for Z made
  of them R = diag(sqrt(lambda_k) * |z_k|) exactly.
* n = 1: r_11 = ||z||_A, q = z / r_11.
* Section 2.1: the column- and row-oriented forms perform the same operations
  in a different order and must agree bit for bit.
* MV counts: 2n (Algorithms 3/4), n (5/7), one block product (6/8).
* Brute force: for m <= 8 the FP64 result matches 60-digit arithmetic.
"""
import numpy as np
import pytest

import oracle
import workloads as W

ALGS = [(v, f) for v in ("naive", "ha", "hp") for f in ("col", "row")]


def identity_csr(m):
    return (np.arange(m + 1, dtype=np.int32), np.arange(m, dtype=np.int32), np.ones(m))


def householder_qr_pos(Z):
    Qh, Rh = np.linalg.qr(Z)
    s = np.sign(np.diag(Rh))
    return Qh * s[None, :], Rh * s[:, None]


@pytest.mark.parametrize("variant,form", ALGS)
def test_identity_equals_householder(variant, form):
    rng = W.rng(7, 100)
    m, n = 60, 12
    Z = np.asfortranarray(rng.standard_normal((m, n)))
    assert np.linalg.cond(Z) < 1e3
    Q, R, info, _, _ = oracle.mgs(identity_csr(m), Z, variant, form)
    assert info == 0
    Qh, Rh = householder_qr_pos(Z)
    assert np.linalg.norm(R - Rh) / np.linalg.norm(Rh) < 1e-14
    assert np.abs(Q - Qh).max() < 1e-13


def _mp_chol_gram(A, Z, dps=50):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    D = W.csr_to_dense(A)
    m, n = Z.shape
    Zm = mp.matrix([[mp.mpf(float(Z[i, j])) for j in range(n)] for i in range(m)])
    Dm = mp.matrix([[mp.mpf(float(D[i, j])) for j in range(m)] for i in range(m)])
    G = Zm.T * Dm * Zm
    L = mp.cholesky(G)
    return np.array([[float(L[j, i]) for j in range(n)] for i in range(n)])  # upper factor R = L^T


@pytest.mark.parametrize("variant,form", ALGS)
def test_R_is_cholesky_of_gram(variant, form):
    A = W.banded_spd_csr(40, 3, W.rng(11, 101))
    Z = np.asfortranarray(W.rng(11, 102).standard_normal((40, 6)))
    Rref = _mp_chol_gram(A, Z)
    Q, R, info, _, _ = oracle.mgs(A, Z, variant, form)
    assert info == 0
    assert np.linalg.norm(R - Rref) / np.linalg.norm(Rref) < 1e-13
    # Q = Z R^{-1} (exact in exact arithmetic)
    Qref = np.linalg.solve(Rref.T, Z.T).T
    assert np.abs(Q - Qref).max() < 1e-12 * np.abs(Qref).max()


def test_chol_gram_long_double_matches_mpmath():
    A = W.banded_spd_csr(30, 4, W.rng(12, 103))
    Z = np.asfortranarray(W.rng(12, 104).standard_normal((30, 5)))
    Rref = _mp_chol_gram(A, Z)
    Rld, info = oracle.chol_gram(A, Z)
    assert info == 0
    assert np.linalg.norm(Rld - Rref) / np.linalg.norm(Rref) < 1e-15


@pytest.mark.parametrize("variant,form", ALGS)
def test_tridiag_sine_eigenvectors_closed_form(variant, form):
    m, n = 64, 6
    A = W.tridiag_csr(m)
    t = np.arange(1, m + 1)
    ks = np.array([1, 3, 4, 10, 20, 33])
    U = np.sqrt(2.0 / (m + 1)) * np.sin(np.outer(t, ks) * np.pi / (m + 1))  # orthonormal eigenvectors
    lam = 2.1 - 2.0 * np.cos(ks * np.pi / (m + 1))
    scale = np.array([1.0, 2.0, 0.5, 3.0, 1.5, 0.25])
    Z = np.asfortranarray(U * scale[None, :])
    Q, R, info, _, _ = oracle.mgs(A, Z, variant, form)
    assert info == 0
    Rexp = np.diag(np.sqrt(lam) * scale)
    assert np.abs(R - Rexp).max() < 1e-13 * np.abs(Rexp).max()
    Qexp = U / np.sqrt(lam)[None, :]
    assert np.abs(Q - Qexp).max() < 1e-13 * np.abs(Qexp).max()


@pytest.mark.parametrize("variant,form", ALGS)
def test_single_column(variant, form):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    A = W.banded_spd_csr(25, 2, W.rng(13, 105))
    z = W.rng(13, 106).standard_normal((25, 1))
    Q, R, info, _, _ = oracle.mgs(A, z, variant, form)
    D = W.csr_to_dense(A)
    s = mp.fsum(mp.mpf(float(z[i, 0])) * mp.mpf(float(D[i, j])) * mp.mpf(float(z[j, 0]))
                for i in range(25) for j in range(25))
    r = mp.sqrt(s)
    assert info == 0
    assert abs(R[0, 0] - float(r)) <= 2e-16 * float(r)
    assert np.abs(Q[:, 0] - z[:, 0] / float(r)).max() <= 4e-16 * np.abs(z).max() / float(r)


@pytest.mark.parametrize("variant", ["naive", "ha", "hp"])
def test_col_and_row_forms_bitwise_equal(variant):
    for (A, Z) in [W.tridiag(300, 9), W.banded(200, 17, seed=5), W.poisson2d(side=12, n=10, lo_exp=-4)]:
        Qc, Rc, ic, _, _ = oracle.mgs(A, Z, variant, "col")
        Qr, Rr, ir, _, _ = oracle.mgs(A, Z, variant, "row")
        assert ic == ir == 0
        assert np.array_equal(Qc, Qr) and np.array_equal(Rc, Rr)


@pytest.mark.parametrize("variant,form,expect", [("naive", "col", 2), ("naive", "row", 2), ("ha", "col", 1),
                                                 ("ha", "row", 1), ("hp", "col", 0), ("hp", "row", 0)])
def test_mv_counts(variant, form, expect):
    A, Z = W.tridiag(100, 7)
    _, _, info, _, mv = oracle.mgs(A, Z, variant, form)
    assert info == 0
    assert mv == (expect * 7 if expect else 1)


def _mp_mgs_naive(A, Z, dps=60):
    """Algorithm 3 in 60-digit arithmetic (rounding-level reference)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    D = W.csr_to_dense(A)
    m, n = Z.shape
    Am = mp.matrix([[mp.mpf(float(D[i, j])) for j in range(m)] for i in range(m)])
    z = [mp.matrix([mp.mpf(float(Z[i, j])) for i in range(m)]) for j in range(n)]
    q, p = [], []
    R = np.zeros((n, n))
    for j in range(n):
        for i in range(j):
            r = (p[i].T * z[j])[0]
            R[i, j] = float(r)
            z[j] = z[j] - r * q[i]
        x = Am * z[j]
        rjj = mp.sqrt((z[j].T * x)[0])
        R[j, j] = float(rjj)
        q.append(z[j] / rjj)
        p.append(Am * q[j])
    Q = np.array([[float(q[j][i]) for j in range(n)] for i in range(m)])
    return Q, R


@pytest.mark.parametrize("m,n", [(1, 1), (3, 2), (6, 6), (8, 5)])
@pytest.mark.parametrize("variant", ["naive", "ha", "hp"])
def test_bruteforce_high_precision(m, n, variant):
    A = W.banded_spd_csr(m, 2, W.rng(14, 107, m))
    Z = np.asfortranarray(W.rng(14, 108, m).standard_normal((m, n)) + 2 * np.eye(m, n))
    Qm, Rm = _mp_mgs_naive(A, Z)
    Q, R, info, _, _ = oracle.mgs(A, Z, variant, "row")
    assert info == 0
    cond = np.linalg.cond(Rm)
    assert np.abs(R - Rm).max() <= 1e-14 * cond * np.abs(Rm).max()
    assert np.abs(Q - Qm).max() <= 1e-14 * cond * np.abs(Qm).max()


@pytest.mark.parametrize("variant,form", ALGS)
def test_invariants(variant, form):
    A, Z = W.banded(500, 24, seed=9)
    Q, R, info, _, _ = oracle.mgs(A, Z, variant, form)
    assert info == 0
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) > 0)
    assert oracle.repr_error(Z, Q, R) < 1e-15
    assert oracle.orth_loss(A, Q) < 1e-13


@pytest.mark.parametrize("variant,form", ALGS)
def test_breakdown_reporting(variant, form):
    m, n = 30, 4
    # Not SPD: a negative diagonal makes z_1^T A z_1 negative for z_1 = e_1.
    rowptr, col, val = identity_csr(m)
    val = val.copy()
    val[0] = -1.0
    Z = np.asfortranarray(np.eye(m, n))
    _, _, info, kind, _ = oracle.mgs((rowptr, col, val), Z, variant, form)
    assert (info, kind) == (1, 1)
    # A zero column is rank deficient: z_3^T A z_3 = 0 at column 3.
    Z = np.asfortranarray(W.rng(15, 109).standard_normal((m, n)))
    Z[:, 2] = 0.0
    _, _, info, kind, _ = oracle.mgs(identity_csr(m), Z, variant, form)
    assert (info, kind) == (3, 1)
    # NaN is reported as non-finite.
    Z[:, 2] = 1.0
    Z[5, 1] = np.nan
    _, _, info, kind, _ = oracle.mgs(identity_csr(m), Z, variant, form)
    assert (info, kind) == (2, 2)


def test_metric_helpers_against_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    A = W.banded_spd_csr(12, 2, W.rng(16, 110))
    Z = np.asfortranarray(W.rng(16, 111).standard_normal((12, 4)))
    Q, R, *_ = oracle.mgs(A, Z, "naive", "col")
    Q = Q + 1e-9 * W.rng(16, 112).standard_normal(Q.shape)  # make both errors clearly non-zero
    Q = np.asfortranarray(Q)
    D = W.csr_to_dense(A)
    Qm = mp.matrix(Q.tolist())
    Dm = mp.matrix(D.tolist())
    Zm = mp.matrix(Z.tolist())
    Rm = mp.matrix(R.tolist())
    E = Zm - Qm * Rm
    ref_repr = mp.sqrt(mp.fsum(E[i, j] ** 2 for i in range(12) for j in range(4))) / \
        mp.sqrt(mp.fsum(Zm[i, j] ** 2 for i in range(12) for j in range(4)))
    G = Qm.T * Dm * Qm - mp.eye(4)
    ref_loss = mp.sqrt(mp.fsum(G[i, j] ** 2 for i in range(4) for j in range(4)))
    assert abs(oracle.repr_error(Z, Q, R) - float(ref_repr)) <= 1e-12 * float(ref_repr)
    assert abs(oracle.orth_loss(A, Q) - float(ref_loss)) <= 1e-12 * float(ref_loss)
