"""The multi-core build of the oracle (``oracle/mgs_oracle_par.c``) against the
single-thread oracle.

The multi-core build performs the operations of the row-oriented Algorithms
4, 7 and 8 in the same order as ``mgs_oracle.c`` (independent rows and
columns on different threads, the one cross-row sum z_i^T x_i on one thread),
so its Q, R, breakdown column and kind must equal the single-thread oracle's
bit for bit, whatever the thread count.  The single-thread oracle is itself
pinned by ``test_oracle_pins.py``; this pin carries those pins over.
"""
import numpy as np
import pytest

import oracle
import workloads as W

CASES = {
    "tridiag_1x1": lambda: W.tridiag(1, 1),
    "tridiag_17x17": lambda: W.tridiag(17, 17),
    "tridiag_500x9": lambda: W.tridiag(500, 9),
    "banded_3001x40": lambda: W.banded(3001, 40, seed=11),
    "poisson2d_48_n16": lambda: W.poisson2d(side=48, n=16),
    "varcoef3d_14_n24": lambda: W.varcoef3d(side=14, n=24),
    "denseband_1500x12": lambda: W.denseband(1500, 12, hb=60),
}


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
@pytest.mark.parametrize("variant", ["naive", "ha", "hp"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_par_equals_single_thread_bitwise(case, variant, threads):
    A, Z = CASES[case]()
    Qs, Rs, info_s, kind_s, _ = oracle.mgs(A, Z, variant, "row")
    Qp, Rp, info_p, kind_p = oracle.mgs_par(A, Z, variant, threads=threads)
    assert (info_p, kind_p) == (info_s, kind_s)
    assert np.array_equal(Rp, Rs)
    assert np.array_equal(Qp, Qs)


@pytest.mark.parametrize("variant", ["naive", "ha", "hp"])
def test_par_breakdown_matches(variant):
    # Column 3 is a combination of columns 0 and 1: z_3^T x_3 vanishes up to
    # rounding, so both builds must stop at the same column with the same kind.
    A, Z = W.banded(400, 6, seed=2)
    Z = np.asfortranarray(Z.copy())
    Z[:, 3] = 2.0 * Z[:, 0] - Z[:, 1]
    Z[:, 5] = np.nan
    Qs, Rs, info_s, kind_s, _ = oracle.mgs(A, Z, variant, "row")
    Qp, Rp, info_p, kind_p = oracle.mgs_par(A, Z, variant, threads=4)
    assert info_s > 0
    assert (info_p, kind_p) == (info_s, kind_s)
    cols = info_s - 1
    assert np.array_equal(Rp[:, :cols], Rs[:, :cols])
    assert np.array_equal(Qp[:, :cols], Qs[:, :cols])


def test_par_reports_threads():
    assert oracle.par_threads(3) == 3 or oracle.par_threads() == 1  # 1: built without OpenMP
    oracle.par_threads(1)
