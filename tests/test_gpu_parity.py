"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Gates (floating point, from the paper's error analysis, Section 3):
  representation  ||Z - QR||_F / ||Z||_F  <= max(1e-13, 10 x oracle's value)
  A-orthogonality ||I - Q^T A Q||_F       <= max(1e-12, 10 x oracle's value)
  R               ||R - R_oracle||_F / ||R||_F <= 1e-10  when kappa(Z) <= 1e3
  element-wise    |Q - Q_oracle| <= 1e-9 * kappa(R) * max|Q_oracle|, likewise R
Both sides run the same algorithm (naive/HA/HP, right-looking); they differ only
in rounding (fused multiply-add, reduction tree, reciprocal scaling).
"""
import numpy as np
import pytest

import oracle
import workloads as W

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
    rowptr, col, val = A
    Ad = (torch.from_numpy(np.ascontiguousarray(rowptr)).to(d), torch.from_numpy(np.ascontiguousarray(col)).to(d),
          torch.from_numpy(np.ascontiguousarray(val)).to(d))
    Zd = torch.from_numpy(np.ascontiguousarray(np.asarray(Z).T)).to(d).T
    return Ad, Zd


def gpu_qr(h, A, Z, variant):
    Ad, Zd = to_dev(A, Z)
    Q, R = h.qr(Ad, Zd, variant)
    st, info = h.info()
    return Q.cpu().numpy(), R.cpu().numpy(), st, info


def check_parity(A, Z, variant, Q, R, well_conditioned=True):
    Qo, Ro, info, _, _ = oracle.mgs(A, Z, variant, "row")
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
    return rep_g, loss_g


SMALL_CASES = {
    "tridiag_1x1": lambda: W.tridiag(1, 1),
    "tridiag_2x2": lambda: W.tridiag(2, 2),
    "tridiag_3x1": lambda: W.tridiag(3, 1),
    "tridiag_17x3": lambda: W.tridiag(17, 3),
    "tridiag_100x16": lambda: W.tridiag(100, 16),
    "tridiag_257x33": lambda: W.tridiag(257, 33),
    "tridiag_4096x16": lambda: W.tridiag(4096, 16),
    "tridiag_5003x7": lambda: W.tridiag(5003, 7),
    "banded_777x20": lambda: W.banded(777, 20, seed=3),
    "banded_3000x64": lambda: W.banded(3000, 64, seed=4),
    "banded_20011x40": lambda: W.banded(20011, 40, seed=5),
    "varcoef3d_12": lambda: W.varcoef3d(side=12, n=24),
    # long rows (warp-per-row MVs): 201 and 389 nonzeros per row
    "denseband_2000x24": lambda: W.denseband(2000, 24, hb=100),
    "denseband_9180x50": lambda: W.denseband(),
}


@pytest.mark.parametrize("case", sorted(SMALL_CASES))
@pytest.mark.parametrize("variant", VARIANTS)
def test_parity_small(handle, case, variant):
    A, Z = SMALL_CASES[case]()
    Q, R, st, info = gpu_qr(handle, A, Z, variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check_parity(A, Z, variant, Q, R)


@pytest.mark.parametrize("variant", VARIANTS)
def test_parity_graded_poisson(handle, variant):
    # kappa(Z) = 1e6: HA/HP accuracy stress at a size the oracle finishes quickly.
    A, Z = W.poisson2d(side=48, n=32)
    Q, R, st, info = gpu_qr(handle, A, Z, variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check_parity(A, Z, variant, Q, R, well_conditioned=False)


@pytest.mark.parametrize("variant", VARIANTS)
def test_parity_dense_exp2(handle, variant):
    # Section 4.2 family, case 2 (worst case), moderate conditioning.
    Ad, Z, _ = W.exp2_problem(4.0, 2.0, case=2)
    A = W.dense_csr(Ad)
    Q, R, st, info = gpu_qr(handle, A, Z, variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check_parity(A, Z, variant, Q, R)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("max_ctas,chunk", [(1, 32), (3, 256), (7, 4096), (2, 96)])
def test_parity_forced_tiling(handle, variant, max_ctas, chunk):
    """Few CTAs and small chunks: many chunks per CTA, ragged last chunk."""
    A, Z = W.banded(5003, 12, seed=6)
    handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, max_ctas)
    handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, chunk)
    try:
        Q, R, st, info = gpu_qr(handle, A, Z, variant)
    finally:
        handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, 0)
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 0)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check_parity(A, Z, variant, Q, R)


@pytest.mark.parametrize("variant", VARIANTS)
def test_deterministic(handle, variant):
    A, Z = W.banded(40000, 24, seed=7)
    Q1, R1, st1, _ = gpu_qr(handle, A, Z, variant)
    Q2, R2, st2, _ = gpu_qr(handle, A, Z, variant)
    assert st1 == st2 == mgsa.MGSA_OK
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2)


@pytest.mark.parametrize("variant", VARIANTS)
def test_breakdown_and_recovery(handle, variant):
    m, n = 300, 5
    rowptr = np.arange(m + 1, dtype=np.int32)
    col = np.arange(m, dtype=np.int32)
    val = np.ones(m)
    val[0] = -1.0
    Z = np.asfortranarray(np.eye(m, n))
    _, _, st, info = gpu_qr(handle, (rowptr, col, val), Z, variant)
    assert (st, info) == (mgsa.MGSA_ERR_BREAKDOWN, 1)
    Z = np.asfortranarray(W.rng(3, 200).standard_normal((m, n)))
    Z[:, 2] = 0.0
    _, _, st, info = gpu_qr(handle, W.tridiag_csr(m), Z, variant)
    assert (st, info) == (mgsa.MGSA_ERR_BREAKDOWN, 3)
    Z[:, 2] = 1.0
    Z[7, 1] = np.nan
    _, _, st, info = gpu_qr(handle, W.tridiag_csr(m), Z, variant)
    assert (st, info) == (mgsa.MGSA_ERR_NONFINITE, 2)
    # the handle keeps working after a failure
    A, Z = W.tridiag(m, n)
    Q, R, st, info = gpu_qr(handle, A, Z, variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check_parity(A, Z, variant, Q, R)


def test_invalid_arguments_rejected_before_launch(handle):
    A, Z = W.tridiag(64, 8)
    Ad, Zd = to_dev(A, Z)
    csr = mgsa.make_csr(64, len(A[1]), *Ad)
    Q = torch.empty((8, 64), dtype=torch.float64, device="cuda").T
    R = torch.empty((8, 8), dtype=torch.float64, device="cuda").T
    bad = [
        dict(m=64, n=0, ldz=64, ldq=64, ldr=8),
        dict(m=4, n=8, ldz=64, ldq=64, ldr=8),
        dict(m=64, n=8, ldz=63, ldq=64, ldr=8),
        dict(m=64, n=8, ldz=64, ldq=64, ldr=7),
        dict(m=64, n=mgsa.MGSA_MAX_N + 1, ldz=64, ldq=64, ldr=8),
    ]
    for b in bad:
        st = mgsa.mgsa_qr(handle.h, csr, Zd, b["m"], b["n"], b["ldz"], mgsa.MGSA_HP, Q, b["ldq"], R, b["ldr"])
        assert st == mgsa.MGSA_ERR_INVALID, b
    # Q overlapping Z without being Z itself (Q == Z runs in place, tests/test_gpu_inplace.py)
    buf = torch.zeros(9 * 64, dtype=torch.float64, device="cuda")
    Zb = buf[: 8 * 64].view(8, 64).T
    Zb.copy_(Zd)
    Qs = buf[32: 32 + 8 * 64].view(8, 64).T
    st = mgsa.mgsa_qr(handle.h, csr, Zb, 64, 8, 64, mgsa.MGSA_HP, Qs, 64, R, 8)
    assert st == mgsa.MGSA_ERR_INVALID
    # A->m mismatch
    csr_bad = mgsa.make_csr(65, len(A[1]), *Ad)
    st = mgsa.mgsa_qr(handle.h, csr_bad, Zd, 64, 8, 64, mgsa.MGSA_HP, Q, 64, R, 8)
    assert st == mgsa.MGSA_ERR_INVALID
    assert mgsa.mgsa_qr(handle.h, csr, Zd, 64, 8, 64, 7, Q, 64, R, 8) == mgsa.MGSA_ERR_INVALID


@pytest.mark.parametrize("variant", VARIANTS)
def test_leading_dimensions(handle, variant):
    """Z, Q, R inside larger column-major buffers (ld > m, ld > n)."""
    A, Z = W.banded(1000, 9, seed=8)
    Ad, _ = to_dev(A, Z)
    d = torch.device("cuda")
    Zbig = torch.full((9, 1037), 7.0, dtype=torch.float64, device=d)
    Zbig[:, :1000] = torch.from_numpy(np.ascontiguousarray(Z.T)).to(d)
    Qbig = torch.full((9, 1100), -3.0, dtype=torch.float64, device=d)
    Rbig = torch.full((9, 11), -5.0, dtype=torch.float64, device=d)
    csr = mgsa.make_csr(1000, len(A[1]), *Ad)
    st = mgsa.mgsa_qr(handle.h, csr, Zbig, 1000, 9, 1037, mgsa.VARIANTS[variant], Qbig, 1100, Rbig, 11)
    assert st == mgsa.MGSA_OK
    assert handle.info() == (mgsa.MGSA_OK, 0)
    Qb, Rb = Qbig.cpu().numpy(), Rbig.cpu().numpy()
    assert np.all(Qb[:, 1000:] == -3.0) and np.all(Rb[:, 9:] == -5.0)
    check_parity(A, Z, variant, np.asfortranarray(Qb[:, :1000].T), np.asfortranarray(Rb[:, :9].T))


@pytest.mark.parametrize("variant", VARIANTS)
def test_host_entry_point_matches_device(handle, variant):
    A, Z = W.banded(2500, 13, seed=9)
    Qd, Rd, st, _ = gpu_qr(handle, A, Z, variant)
    Qh = np.zeros((2500, 13), order="F")
    Rh = np.zeros((13, 13), order="F")
    rowptr, col, val = A
    st, info = mgsa.mgsa_qr_host(handle.h, rowptr, col, val, len(col), np.asfortranarray(Z), 2500, 13, 2500,
                                 mgsa.VARIANTS[variant], Qh, 2500, Rh, 13)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    assert np.array_equal(Qh, Qd) and np.array_equal(Rh, Rd)


@pytest.mark.parametrize("variant", VARIANTS)
def test_parity_long_rows_multi_chunk(handle, variant):
    """Warp-per-row MVs outside resident mode (two CTAs, several chunks each)."""
    A, Z = W.denseband(9180, 20)
    handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, 2)
    handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 1024)
    try:
        Q, R, st, info = gpu_qr(handle, A, Z, variant)
    finally:
        handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, 0)
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 0)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check_parity(A, Z, variant, Q, R)


@pytest.mark.parametrize("variant", VARIANTS + ["cgs_naive", "cgs_ha", "cgs_hp"])
@pytest.mark.parametrize("min_rows,chunk", [(0, 0), (32, 0), (0, 64)])
def test_max_width_closed_form(handle, variant, min_rows, chunk):
    """The widest QR the library takes, n = MGSA_MAX_N = 2048 with m = n.  Z
    is the whole sine eigenbasis U of tridiag(-1, 2.1, -1) with columns scaled
    by s_k, so Z^T A Z = diag(s_k^2 lambda_k): R = diag(s_k sqrt(lambda_k))
    and Q = U diag(1 / sqrt(lambda_k)) exactly (the closed form the oracle is
    pinned to at small sizes; the oracle's own HP run at this size is within
    1e-13 (R) and 2.5e-13 (Q) of it, relative to the largest entry, and so is
    its CGS-HA run).  MGS and CGS forms; 16 CTAs (default), 64 CTAs (every
    CTA then sums about 32 entries of each row of R), and pivots staged in
    64-row chunks."""
    m = n = mgsa.MGSA_MAX_N
    A = W.tridiag_csr(m)
    t = np.arange(1, m + 1)
    ks = np.arange(1, n + 1)
    U = np.sqrt(2.0 / (m + 1)) * np.sin(np.outer(t, ks) * np.pi / (m + 1))
    lam = 2.1 - 2.0 * np.cos(ks * np.pi / (m + 1))
    scale = 1.0 + (ks % 7) / 4.0
    Z = U * scale[None, :]
    handle.set_param(mgsa.MGSA_PARAM_MIN_ROWS_PER_CTA, min_rows)
    handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, chunk)
    try:
        Q, R, st, info = gpu_qr(handle, A, Z, variant)
    finally:
        handle.set_param(mgsa.MGSA_PARAM_MIN_ROWS_PER_CTA, 0)
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 0)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    Rexp = np.diag(np.sqrt(lam) * scale)
    Qexp = U / np.sqrt(lam)[None, :]
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) > 0)
    assert np.abs(R - Rexp).max() <= 1e-11 * np.abs(Rexp).max()
    assert np.abs(Q - Qexp).max() <= 1e-11 * np.abs(Qexp).max()


ALL_FORMS = VARIANTS + ["cgs_naive", "cgs_ha", "cgs_hp"]


def oracle_form(A, Z, form):
    if form.startswith("cgs_"):
        return oracle.cgs(A, Z, form[4:], "col")
    return oracle.mgs(A, Z, form, "row")


@pytest.mark.parametrize("form", ALL_FORMS)
def test_identity_matches_householder(handle, form):
    """A = I: the A-inner product is the Euclidean one, so every form computes
    the Householder QR of Z with the signs fixed so that diag(R) > 0 (numpy's
    LAPACK QR, not the oracle)."""
    m, n = 3001, 40
    A = (np.arange(m + 1, dtype=np.int32), np.arange(m, dtype=np.int32), np.ones(m))
    Z = W.rng(6, 301).standard_normal((m, n))
    Q, R, st, info = gpu_qr(handle, A, Z, form)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    Qh, Rh = np.linalg.qr(Z)
    s = np.sign(np.diag(Rh))
    Qh, Rh = Qh * s[None, :], Rh * s[:, None]
    assert np.abs(R - Rh).max() <= 1e-12 * np.abs(Rh).max()
    assert np.abs(Q - Qh).max() <= 1e-12 * np.abs(Qh).max()


@pytest.mark.parametrize("form", ALL_FORMS)
def test_empty_rows_and_empty_matrix(handle, form):
    """CSR rows without entries.  A = diag(d) with every other row empty is
    positive definite on the even rows, where Z lives: the QR succeeds and
    matches the oracle's.  A with no entries at all (nnz = 0, no column or
    value array) breaks down at column 1."""
    m, n = 2003, 9
    d = np.where(np.arange(m) % 2 == 0, 1.0 + np.arange(m) / m, 0.0)
    rows = np.nonzero(d)[0]
    rowptr = np.zeros(m + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum(d != 0)
    A = (rowptr, rows.astype(np.int32), d[rows])
    Z = W.rng(6, 302).standard_normal((m, n))
    Z[1::2, :] = 0.0
    Q, R, st, info = gpu_qr(handle, A, Z, form)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    Qo, Ro, oinfo, _, _ = oracle_form(A, Z, form)
    assert oinfo == 0
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10
    assert np.abs(Q - Qo).max() <= 1e-10 * np.abs(Qo).max()
    assert np.all(Q[1::2, :] == 0.0)
    A0 = (np.zeros(m + 1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    _, _, st, info = gpu_qr(handle, A0, Z, form)
    assert (st, info) == (mgsa.MGSA_ERR_BREAKDOWN, 1)
