"""Pins of the oracle's classical Gram-Schmidt (CGS-naive / HA / HP).

Section 2.3 extends the n-MV idea to CGS; Section 3.3 gives its recurrences:
MGS's with z_j^{(i-1)} replaced by z_j^{(0)} in r_ij.  What fixes the oracle:
  * the column and row forms perform the same operations on every column in
    the same order, so they agree bit for bit (as for MGS, Section 2.1);
  * with n <= 2 every r_ij is taken against z_j^{(0)} = z_j^{(i-1)} anyway,
    so CGS is MGS bit for bit (MGS is pinned in test_oracle_pins.py);
  * in exact arithmetic R is the Cholesky factor of Z^T A Z and Q = Z R^{-1};
  * MV counts: naive 2n, HA n, HP one block product;
  * Section 4.2: the loss of A-orthogonality of CGS grows quadratically with
    kappa(A^{1/2} Z), against linearly for MGS; Section 3.3: CGS-HA loses
    about as much A-orthogonality as CGS-naive.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from exp2_grid import LOGS

VARIANTS = ["naive", "ha", "hp"]


def small_problems():
    out = [W.tridiag(40, 6), W.banded(300, 9, seed=11), W.varcoef3d(side=6, n=10)]
    A = W.banded_spd_csr(80, 4, W.rng(31, 1))
    out.append((A, np.asfortranarray(W.rng(31, 2).standard_normal((80, 12)))))
    return out


@pytest.mark.parametrize("variant", VARIANTS)
def test_col_equals_row_bitwise(variant):
    for A, Z in small_problems():
        Qc, Rc, ic, _, mc = oracle.cgs(A, Z, variant, "col")
        Qr, Rr, ir, _, mr = oracle.cgs(A, Z, variant, "row")
        assert ic == ir == 0 and mc == mr
        assert np.array_equal(Qc, Qr) and np.array_equal(Rc, Rr)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("form", ["col", "row"])
def test_two_columns_equal_mgs(variant, form):
    for A, Z in small_problems():
        for n in (1, 2):
            Qc, Rc, ic, kc, mc = oracle.cgs(A, Z[:, :n], variant, form)
            Qm, Rm, im, km, mm = oracle.mgs(A, Z[:, :n], variant, form)
            assert (ic, kc, mc) == (im, km, mm) == (0, 0, mm)
            assert np.array_equal(Qc, Qm) and np.array_equal(Rc, Rm)


@pytest.mark.parametrize("variant", VARIANTS)
def test_cholesky_closed_form(variant):
    """Well-conditioned Z: R = chol(Z^T A Z), Z = QR, Q^T A Q = I to rounding."""
    for A, Z in small_problems():
        Q, R, info, _, _ = oracle.cgs(A, Z, variant, "col")
        assert info == 0
        Rc, ok = oracle.chol_gram(A, Z)
        assert ok == 0
        assert np.linalg.norm(R - Rc) / np.linalg.norm(Rc) <= 1e-12
        assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
        assert oracle.repr_error(Z, Q, R) <= 1e-15
        assert oracle.orth_loss(A, Q) <= 1e-12


@pytest.mark.parametrize("variant,expect", [("naive", lambda n: 2 * n), ("ha", lambda n: n), ("hp", lambda n: 1)])
def test_mv_counts(variant, expect):
    A, Z = W.banded(200, 7, seed=12)
    for form in ("col", "row"):
        assert oracle.cgs(A, Z, variant, form)[4] == expect(7)


@pytest.mark.parametrize("variant", VARIANTS)
def test_breakdown_reports_column(variant):
    A, Z = W.tridiag(50, 5)
    Z = Z.copy()
    Z[:, 3] = 0.0
    for form in ("col", "row"):
        _, _, info, kind, _ = oracle.cgs(A, Z, variant, form)
        assert (info, kind) == (4, 1)
    Z[0, 1] = np.nan
    _, _, info, kind, _ = oracle.cgs(A, Z, variant, "col")
    assert (info, kind) == (2, 2)


def loss_curve(fn, variant, log_kA, lzs, case=1):
    out = []
    for lz in lzs:
        Ad, Z, _ = W.exp2_problem(log_kA, lz, case)
        A = W.dense_csr(Ad)
        Q, _, info, _, _ = fn(A, Z, variant, "row")
        out.append(oracle.orth_loss(A, Q) if info == 0 else np.inf)
    return np.array(out)


LZ = LOGS[(LOGS >= 1.0) & (LOGS <= 6.0)]


@pytest.mark.parametrize("variant", VARIANTS)
def test_loss_quadratic_in_kappa(variant):
    """Section 4.2: CGS's loss grows like kappa(A^{1/2} Z)^2, MGS's like
    kappa(A^{1/2} Z) (case 1, kappa(A) = 10^2, while the loss is below 1)."""
    cg = loss_curve(oracle.cgs, variant, 2.0, LZ)
    mg = loss_curve(oracle.mgs, variant, 2.0, LZ)
    assert np.all(np.isfinite(cg)) and np.all(cg < 1e-2)
    s_cgs = np.polyfit(LZ, np.log10(cg), 1)[0]
    s_mgs = np.polyfit(LZ, np.log10(mg), 1)[0]
    assert 1.7 <= s_cgs <= 2.3, s_cgs
    assert 0.8 <= s_mgs <= 1.2, s_mgs
    assert cg[-1] > 100 * mg[-1]


def test_ha_loss_close_to_naive():
    """Section 3.3: CGS-HA is expected to lose about as much A-orthogonality
    as CGS-naive.  Read on the Section 4.2 grid (every other kappa(A) and
    kappa(A^{1/2} Z), both cases, where the naive loss is below 1e-2): the
    geometric mean of loss(HA) / loss(naive) lies in [1/2, 2] and no single
    problem differs by more than a factor 30 either way."""
    for case in (1, 2):
        ratios = []
        for la in LOGS[::2]:
            ln = loss_curve(oracle.cgs, "naive", la, LOGS[::2], case)
            lh = loss_curve(oracle.cgs, "ha", la, LOGS[::2], case)
            ok = np.isfinite(ln) & np.isfinite(lh) & (ln < 1e-2)
            ratios.extend(lh[ok] / ln[ok])
        ratios = np.array(ratios)
        assert len(ratios) >= 50
        gmean = np.exp(np.mean(np.log(ratios)))
        assert 0.5 <= gmean <= 2.0, (case, gmean)
        assert ratios.min() >= 1 / 30 and ratios.max() <= 30, (case, ratios.min(), ratios.max())
