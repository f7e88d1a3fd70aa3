"""Successive orthogonalisation in the oracle (Section 2.1's column-oriented
MGS).  Pins: with k = 0 it is Algorithm 3/5/6 (bitwise equal to the column
form); appending n columns to the result of the first k performs the
operations of one run over all k + n columns (bitwise); and the appended
factorisation satisfies the invariants of eq. (1) for the concatenation."""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("variant", ["naive", "ha", "hp"])
def test_append_with_no_old_columns_is_the_column_algorithm(variant):
    A, Z = W.banded(400, 12, seed=31)
    Q, P, R, info, _, mv = oracle.mgs_append(A, None, None, Z, variant)
    Qc, Rc, infoc, _, mvc = oracle.mgs(A, Z, variant, "col")
    assert info == infoc == 0 and mv == mvc
    assert np.array_equal(Q, Qc) and np.array_equal(R, Rc)


@pytest.mark.parametrize("variant", ["naive", "ha", "hp"])
@pytest.mark.parametrize("k", [1, 5, 13])
def test_append_equals_one_run_over_all_columns(variant, k):
    A, Zall = W.banded(500, 20, seed=32)
    Q1, P1, R1, info1, _, _ = oracle.mgs_append(A, None, None, Zall[:, :k], variant)
    Q2, P2, R2, info2, _, _ = oracle.mgs_append(A, Q1, P1, Zall[:, k:], variant)
    Qf, Pf, Rf, infof, _, _ = oracle.mgs_append(A, None, None, Zall, variant)
    assert info1 == info2 == infof == 0
    assert np.array_equal(Q2, Qf[:, k:]) and np.array_equal(P2, Pf[:, k:])
    assert np.array_equal(R2, Rf[:, k:])


@pytest.mark.parametrize("variant", ["naive", "ha", "hp"])
def test_append_invariants(variant):
    A, Zall = W.tridiag(300, 16)
    k = 6
    Q1, P1, R1, _, _, _ = oracle.mgs_append(A, None, None, Zall[:, :k], variant)
    Q2, P2, R2, info, _, _ = oracle.mgs_append(A, Q1, P1, Zall[:, k:], variant)
    assert info == 0
    Qall = np.asfortranarray(np.hstack([Q1, Q2]))
    Rall = np.zeros((16, 16))
    Rall[:k, :k] = R1
    Rall[:, k:] = R2
    assert oracle.repr_error(Zall, Qall, Rall) < 1e-15
    assert oracle.orth_loss(A, Qall) < 1e-13
    Rc, _ = oracle.chol_gram(A, Zall)
    assert np.linalg.norm(Rall - Rc) / np.linalg.norm(Rc) < 1e-13
