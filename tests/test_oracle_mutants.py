"""Planted mistakes in the oracle are caught by the pins.

Each mutant build of oracle/mgs_oracle.c (compile-time ORACLE_MUTANT, CPU
only) plants one plausible mistake; at least one pin -- the Cholesky factor
of Z^T A Z, A-orthogonality, or the accuracy statements of Sections 4.2/4.3 --
must reject it for the variant it affects.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from exp2_grid import check_paper_claims, problems
from oracle import build as obuild

MUTANTS = {1: ["ha"], 2: ["hp"], 3: ["naive", "ha", "hp"], 4: ["naive", "ha", "hp"]}


def mutant_lib(k):
    out = os.path.join(obuild.OUT_DIR, f"libmgsa_oracle_mutant{k}.so")
    return oracle.load(obuild.build(extra_flags=[f"-DORACLE_MUTANT={k}"], out=out))


def pins_pass(lib, variant, claims: bool = True) -> bool:
    A = W.banded_spd_csr(60, 3, W.rng(21, 400))
    Z = np.asfortranarray(W.rng(21, 401).standard_normal((60, 8)))
    Rc, _ = oracle.chol_gram(A, Z)
    Q, R, info, _, _ = oracle.mgs(A, Z, variant, "row", lib=lib)
    if info != 0 or np.linalg.norm(R - Rc) / np.linalg.norm(Rc) > 1e-12:
        return False
    if oracle.orth_loss(A, Q) > 1e-12:
        return False
    if not claims:
        return True
    rows = []
    for case, la, lz, A2, Z2 in problems(step=3):
        loss = {}
        for v in ("naive", "ha", "hp"):
            Q2, _, inf2, _, _ = oracle.mgs(A2, Z2, v, "row", lib=lib)
            loss[v] = oracle.orth_loss(A2, Q2) if inf2 == 0 else np.inf
        rows.append((case, la, lz, loss))
    try:
        check_paper_claims(rows)
    except AssertionError:
        return False
    return True


def test_unmutated_oracle_passes_the_same_pins():
    for v in ("naive", "ha", "hp"):
        assert pins_pass(oracle.load(), v)


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_planted_mistake_is_caught(k):
    lib = mutant_lib(k)
    for v in MUTANTS[k]:
        assert not pins_pass(lib, v), (k, v)
    # The mistakes that break the factorisation itself are caught by the
    # Cholesky / A-orthogonality pins alone, variant by variant.  Mutant 2 is
    # different: without eq. (tec2)'s recurrence, x_i = A z_i^{(0)} still gives
    # the right r_ii and r_ij in exact arithmetic (z_i^{(i-1)} is A-orthogonal
    # to every earlier q_k), so only the accuracy statements of Sections
    # 4.2/4.3 reveal it.
    if k in (3, 4):
        for v in MUTANTS[k]:
            assert not pins_pass(lib, v, claims=False), (k, v)


def cgs_pins_pass(lib, variant) -> bool:
    """The CGS pins of test_oracle_cgs.py: the Cholesky factor and the
    quadratic growth of the loss with kappa(A^{1/2} Z) (Section 4.2)."""
    A = W.banded_spd_csr(60, 3, W.rng(21, 400))
    Z = np.asfortranarray(W.rng(21, 401).standard_normal((60, 8)))
    Rc, _ = oracle.chol_gram(A, Z)
    _, R, info, _, _ = oracle.cgs(A, Z, variant, "col", lib=lib)
    if info != 0 or np.linalg.norm(R - Rc) / np.linalg.norm(Rc) > 1e-12:
        return False
    lzs = np.arange(2, 13) * 0.5
    losses = []
    for lz in lzs:
        Ad, Z2, _ = W.exp2_problem(2.0, lz, 1)
        A2 = W.dense_csr(Ad)
        Q2, _, inf2, _, _ = oracle.cgs(A2, Z2, variant, "row", lib=lib)
        if inf2 != 0:
            return False
        losses.append(oracle.orth_loss(A2, Q2))
    slope = np.polyfit(lzs, np.log10(losses), 1)[0]
    return 1.7 <= slope <= 2.3


def test_unmutated_cgs_passes_its_pins():
    for v in ("naive", "ha", "hp"):
        assert cgs_pins_pass(oracle.load(), v)


def test_cgs_turned_mgs_is_caught():
    """Mutant 5 takes r_ij against the working column: the result is MGS,
    exact in exact arithmetic, so only the loss growth can tell."""
    lib = mutant_lib(5)
    for v in ("naive", "ha", "hp"):
        assert not cgs_pins_pass(lib, v), v
