"""Parity of the left-looking CGS kernels (MGSA_CGS_NAIVE / HA / HP) with the
oracle's classical Gram-Schmidt (Section 2.3; recurrences of Section 3.3).

Gates, as for MGS (Section 3): representation error and loss of
A-orthogonality within 10x the oracle's (floors 1e-13 / 1e-12); for
well-conditioned Z, R within 1e-10 relative and Q, R element-wise within
1e-9 * kappa(R) of their largest entry.  On the Section 4.2 grid the GPU
losses stay within 10x the oracle's and grow quadratically with
kappa(A^{1/2} Z), as the paper states for CGS.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from exp2_grid import LOGS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402

VARIANTS = ["naive", "ha", "hp"]


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    h = mgsa.Handle(0)
    yield h
    h.close()


def to_dev(A, Z):
    d = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(x)).to(d) for x in A)
    Zd = torch.from_numpy(np.ascontiguousarray(np.asarray(Z).T)).to(d).T
    return Ad, Zd


def gpu_cgs(h, A, Z, variant):
    Ad, Zd = to_dev(A, Z)
    Q, R = h.qr(Ad, Zd, "cgs_" + variant)
    st, info = h.info()
    return Q.cpu().numpy(), R.cpu().numpy(), st, info


def check(A, Z, variant, Q, R, well_conditioned=True):
    Qo, Ro, info, _, _ = oracle.cgs(A, Z, variant, "col")
    assert info == 0
    rep_o, rep_g = oracle.repr_error(Z, Qo, Ro), oracle.repr_error(Z, Q, R)
    loss_o, loss_g = oracle.orth_loss(A, Qo), oracle.orth_loss(A, Q)
    assert rep_g <= max(1e-13, 10 * rep_o), (rep_g, rep_o)
    assert loss_g <= max(1e-12, 10 * loss_o), (loss_g, loss_o)
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) > 0)
    if well_conditioned:
        assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10
        kR = np.linalg.cond(Ro)
        assert np.abs(R - Ro).max() <= 1e-9 * kR * np.abs(Ro).max()
        assert np.abs(Q - Qo).max() <= 1e-9 * kR * np.abs(Qo).max()


CASES = {
    "tridiag_1x1": lambda: W.tridiag(1, 1),
    "tridiag_2x2": lambda: W.tridiag(2, 2),
    "tridiag_17x3": lambda: W.tridiag(17, 3),
    "tridiag_257x33": lambda: W.tridiag(257, 33),
    "tridiag_5003x7": lambda: W.tridiag(5003, 7),
    "banded_777x20": lambda: W.banded(777, 20, seed=3),
    "banded_3000x64": lambda: W.banded(3000, 64, seed=4),
    "banded_20011x40": lambda: W.banded(20011, 40, seed=5),
    "banded_9001x130": lambda: W.banded(9001, 130, seed=13),  # more than 64 pivots per pass
    "varcoef3d_12": lambda: W.varcoef3d(side=12, n=24),
    "denseband_2000x24": lambda: W.denseband(2000, 24, hb=100),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("variant", VARIANTS)
def test_cgs_parity(handle, case, variant):
    A, Z = CASES[case]()
    Q, R, st, info = gpu_cgs(handle, A, Z, variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check(A, Z, variant, Q, R)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("max_ctas,chunk", [(1, 32), (3, 256), (7, 4096), (2, 96)])
def test_cgs_staged(handle, variant, max_ctas, chunk):
    """Few CTAs and small chunks: U and F stream each slab chunk by chunk."""
    A, Z = W.banded(5003, 12, seed=6)
    handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, max_ctas)
    handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, chunk)
    try:
        Q, R, st, info = gpu_cgs(handle, A, Z, variant)
    finally:
        handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, 0)
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 0)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check(A, Z, variant, Q, R)


@pytest.mark.parametrize("variant", VARIANTS)
def test_cgs_staged_long_rows(handle, variant):
    A, Z = W.denseband(2000, 24, hb=100)
    handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, 2)
    handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 256)
    try:
        Q, R, st, info = gpu_cgs(handle, A, Z, variant)
    finally:
        handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, 0)
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 0)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check(A, Z, variant, Q, R)


@pytest.mark.parametrize("variant", VARIANTS)
def test_cgs_deterministic(handle, variant):
    A, Z = W.banded(40000, 24, seed=7)
    Q1, R1, st1, _ = gpu_cgs(handle, A, Z, variant)
    Q2, R2, st2, _ = gpu_cgs(handle, A, Z, variant)
    assert st1 == st2 == mgsa.MGSA_OK
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2)


@pytest.mark.parametrize("variant", VARIANTS)
def test_cgs_two_columns_equal_mgs(handle, variant):
    """With two columns CGS and MGS are the same algorithm (r_01 against
    z_1^{(0)} either way): the GPU results agree to rounding."""
    A, Z = W.banded(6000, 2, seed=14)
    Qc, Rc, st, info = gpu_cgs(handle, A, Z, variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    Ad, Zd = to_dev(A, Z)
    Qm, Rm = handle.qr(Ad, Zd, variant)
    assert handle.info() == (mgsa.MGSA_OK, 0)
    assert np.abs(Rc - Rm.cpu().numpy()).max() <= 1e-13 * np.abs(Rc).max()
    assert np.abs(Qc - Qm.cpu().numpy()).max() <= 1e-13 * np.abs(Qc).max()


@pytest.mark.parametrize("variant", VARIANTS)
def test_cgs_breakdown(handle, variant):
    A, Z = W.tridiag(300, 5)
    Z = Z.copy()
    Z[:, 3] = 0.0
    _, _, info_o, kind_o, _ = oracle.cgs(A, Z, variant, "col")
    assert (info_o, kind_o) == (4, 1)
    _, _, st, info = gpu_cgs(handle, A, Z, variant)
    assert (st, info) == (mgsa.MGSA_ERR_BREAKDOWN, 4)
    Z[:, 3] = np.nan
    _, _, st, info = gpu_cgs(handle, A, Z, variant)
    assert (st, info) == (mgsa.MGSA_ERR_NONFINITE, 4)
    A2, Z2 = W.tridiag(300, 5)  # the handle is still usable
    Q, R, st, info = gpu_cgs(handle, A2, Z2, variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check(A2, Z2, variant, Q, R)


@pytest.mark.parametrize("variant", VARIANTS)
def test_cgs_exp2_grid(handle, variant):
    """Section 4.2 problems (m = 100, n = 20): GPU loss within 10x the oracle's
    wherever the oracle's loss is below 1e-2, and quadratic growth with
    kappa(A^{1/2} Z) in case 1."""
    slopes = []
    for la in (1.0, 4.0):
        xs, ys = [], []
        for case in (1, 2):
            for lz in LOGS[::3]:
                Ad, Z, _ = W.exp2_problem(la, lz, case)
                A = W.dense_csr(Ad)
                Qo, _, io, _, _ = oracle.cgs(A, Z, variant, "col")
                lo = oracle.orth_loss(A, Qo) if io == 0 else np.inf
                Q, R, st, info = gpu_cgs(handle, A, Z, variant)
                if lo < 1e-2:
                    assert (st, info) == (mgsa.MGSA_OK, 0), (la, lz, case)
                    lg = oracle.orth_loss(A, Q)
                    assert lg <= max(1e-12, 10 * lo), (la, lz, case, lg, lo)
                    if case == 1 and 1.0 <= lz <= 6.0:
                        xs.append(lz)
                        ys.append(np.log10(lg))
        slopes.append(np.polyfit(xs, ys, 1)[0])
    assert all(1.6 <= s <= 2.4 for s in slopes), slopes


def test_cgs_rejected_where_unsupported(handle):
    """CGS runs through mgsa_qr only: append, batched and no-alloc refuse it."""
    A, Z = W.tridiag(200, 4)
    Ad, Zd = to_dev(A, Z)
    m, n = Z.shape
    csr = mgsa.make_csr(m, A[1].size, *Ad)
    Q = torch.empty((n, m), dtype=torch.float64, device="cuda").T
    R = torch.empty((n, n), dtype=torch.float64, device="cuda").T
    st = mgsa.mgsa_qr_append(handle.h, csr, None, m, None, m, 0, Zd, m, n, m, mgsa.MGSA_CGS_HA, Q, m, None, m, R, n)
    assert st == mgsa.MGSA_ERR_INVALID
    st = mgsa.mgsa_qr_noalloc(csr, Zd, m, n, m, mgsa.MGSA_CGS_HP, Q, m, R, n)
    assert st == mgsa.MGSA_ERR_INVALID
    assert mgsa.mgsa_job_workspace_bytes(m, n, mgsa.MGSA_CGS_HA) == 0
    st = mgsa.mgsa_qr(handle.h, csr, Zd, m, n, m, 6, Q, m, R, n)
    assert st == mgsa.MGSA_ERR_INVALID
