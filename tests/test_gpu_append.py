"""Successive orthogonalisation on the GPU (``mgsa_qr_append``) against the
oracle's column-oriented append (Section 2: the left-looking MGS is the form
that suits orthogonalising new columns against ones already A-orthonormal).

The GPU runs the right-looking sweep over [Qold Z] with the first k pivots
given; the oracle runs Algorithm 3/5/6 column by column.  They agree in exact
arithmetic, so the gates are those of the plain QR (Section 3): representation
error and loss of A-orthogonality within 10x the oracle's (absolute floors
1e-13 / 1e-12); when [Qold Z] is well conditioned, R within 1e-10 relative
and Q, P element-wise within 1e-9 * kappa(R) of the largest entry.
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


def dev_csr(A):
    d = torch.device("cuda")
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)


def dev_cols(M):
    """Column-major float64 device copy of an (m, n) array (None stays None)."""
    if M is None:
        return None
    return torch.from_numpy(np.ascontiguousarray(np.asarray(M, dtype=np.float64).T)).cuda().T


def host(t):
    return None if t is None else t.cpu().numpy()


def gpu_append(h, A, Qo, Po, Z, variant, want_p=True):
    Q, P, R = h.append(dev_csr(A), dev_cols(Qo), dev_cols(Po), dev_cols(Z), variant, want_p=want_p)
    st, info = h.info()
    return host(Q), host(P), host(R), st, info


def full_factors(Qo, Q, R):
    """[Qold Q] and the square R of [Qold Z] = [Qold Q] [[I, R_top], [0, R_bot]]."""
    k = 0 if Qo is None else Qo.shape[1]
    n = Q.shape[1]
    Rf = np.zeros((k + n, k + n))
    Rf[:k, :k] = np.eye(k)
    Rf[:, k:] = R
    Qf = Q if k == 0 else np.hstack([Qo, Q])
    return Qf, Rf


def check_append(A, Qo, Po, Z, variant, Q, P, R, well_conditioned=True):
    Qr, Pr, Rr, info, _, _ = oracle.mgs_append(A, Qo, Po, Z, variant)
    assert info == 0
    Zf = Z if Qo is None else np.hstack([Qo, Z])
    Qf_o, Rf_o = full_factors(Qo, Qr, Rr)
    Qf_g, Rf_g = full_factors(Qo, Q, R)
    rep_o, rep_g = oracle.repr_error(Zf, Qf_o, Rf_o), oracle.repr_error(Zf, Qf_g, Rf_g)
    loss_o, loss_g = oracle.orth_loss(A, Qf_o), oracle.orth_loss(A, Qf_g)
    assert rep_g <= max(1e-13, 10 * rep_o), (rep_g, rep_o)
    assert loss_g <= max(1e-12, 10 * loss_o), (loss_g, loss_o)
    k = 0 if Qo is None else Qo.shape[1]
    assert np.all(np.tril(R[k:], -1) == 0.0) and np.all(np.diag(R[k:]) > 0)
    if well_conditioned:
        assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= 1e-10
        kR = np.linalg.cond(Rf_o)
        assert np.abs(Q - Qr).max() <= 1e-9 * kR * np.abs(Qr).max()
        if P is not None:
            assert np.abs(P - Pr).max() <= 1e-9 * kR * np.abs(Pr).max()
    return rep_g, loss_g


def oracle_basis(A, Z, variant):
    """A-orthonormal (Q, P) from the oracle, to serve as the given columns."""
    Q, P, _, info, _, _ = oracle.mgs_append(A, None, None, Z, variant)
    assert info == 0
    return Q, P


CASES = {
    # (A, Z) generator, k given columns; covers ragged tails, one and many
    # CTAs, resident and long-row (warp-per-row) paths.
    "tridiag_100_k3_n5": (lambda: W.tridiag(100, 8), 3),
    "tridiag_5003_k7_n9": (lambda: W.tridiag(5003, 16), 7),
    "banded_777_k1_n19": (lambda: W.banded(777, 20, seed=3), 1),
    "banded_20011_k16_n24": (lambda: W.banded(20011, 40, seed=5), 16),
    "varcoef3d_12_k8_n16": (lambda: W.varcoef3d(side=12, n=24), 8),
    "denseband_2000_k10_n14": (lambda: W.denseband(2000, 24, hb=100), 10),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("variant", VARIANTS)
def test_append_parity(handle, case, variant):
    gen, k = CASES[case]
    A, Zall = gen()
    Qo, Po = oracle_basis(A, Zall[:, :k], variant)
    Z = Zall[:, k:]
    Q, P, R, st, info = gpu_append(handle, A, Qo, Po, Z, variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    assert R.shape == (Zall.shape[1], Z.shape[1])
    check_append(A, Qo, Po, Z, variant, Q, P, R)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("max_ctas,chunk", [(1, 32), (3, 256), (2, 96)])
def test_append_forced_tiling(handle, variant, max_ctas, chunk):
    """Staged (non-resident) path: given pivots streamed chunk by chunk."""
    A, Zall = W.banded(5003, 12, seed=6)
    k = 5
    Qo, Po = oracle_basis(A, Zall[:, :k], variant)
    handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, max_ctas)
    handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, chunk)
    try:
        Q, P, R, st, info = gpu_append(handle, A, Qo, Po, Zall[:, k:], variant)
    finally:
        handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, 0)
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 0)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check_append(A, Qo, Po, Zall[:, k:], variant, Q, P, R)


@pytest.mark.parametrize("variant", VARIANTS)
def test_append_k0_is_qr(handle, variant):
    """No given columns: the very same sweep as mgsa_qr, bit for bit."""
    A, Z = W.banded(3000, 17, seed=8)
    Q, P, R, st, info = gpu_append(handle, A, None, None, Z, variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    Q2, R2 = handle.qr(dev_csr(A), dev_cols(Z), variant)
    assert handle.info() == (mgsa.MGSA_OK, 0)
    assert np.array_equal(Q, host(Q2)) and np.array_equal(R, host(R2))
    # without P the result is unchanged
    Q3, P3, R3, st, info = gpu_append(handle, A, None, None, Z, variant, want_p=False)
    assert P3 is None and np.array_equal(Q, Q3) and np.array_equal(R, R3)


@pytest.mark.parametrize("variant", VARIANTS)
def test_append_equals_one_qr(handle, variant):
    """QR of Z1, then append Z2 with the returned (Q, P): the same factors as
    one QR of [Z1 Z2] up to rounding (the pivots are the same numbers)."""
    A, Zall = W.banded(9001, 24, seed=9)
    k = 10
    Q1, P1, R1, st, info = gpu_append(handle, A, None, None, Zall[:, :k], variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    Q2, P2, R2, st, info = gpu_append(handle, A, Q1, P1, Zall[:, k:], variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    Qf, Rf = handle.qr(dev_csr(A), dev_cols(Zall), variant)
    assert handle.info() == (mgsa.MGSA_OK, 0)
    Qf, Rf = host(Qf), host(Rf)
    scale = np.abs(Rf).max()
    assert np.abs(R1 - Rf[:k, :k]).max() <= 1e-12 * scale
    assert np.abs(R2 - Rf[:, k:]).max() <= 1e-12 * scale
    assert np.abs(np.hstack([Q1, Q2]) - Qf).max() <= 1e-11 * np.abs(Qf).max()


@pytest.mark.parametrize("variant", VARIANTS)
def test_append_grows_basis(handle, variant):
    """Four appends of 8 columns: the basis stays A-orthonormal and every
    block is represented, as one oracle run over all 32 columns is."""
    A, Zall = W.banded(12000, 32, seed=10)
    Qb = Pb = None
    blocks = []
    for b in range(4):
        Z = Zall[:, 8 * b: 8 * b + 8]
        Q, P, R, st, info = gpu_append(handle, A, Qb, Pb, Z, variant)
        assert (st, info) == (mgsa.MGSA_OK, 0)
        blocks.append(R)
        Qb = Q if Qb is None else np.hstack([Qb, Q])
        Pb = P if Pb is None else np.hstack([Pb, P])
    Rf = np.zeros((32, 32))
    for b, R in enumerate(blocks):
        Rf[: 8 * b + 8, 8 * b: 8 * b + 8] = R
    Qo, Ro, info, _, _ = oracle.mgs(A, Zall, variant, "col")
    assert info == 0
    assert oracle.orth_loss(A, Qb) <= max(1e-12, 10 * oracle.orth_loss(A, Qo))
    assert oracle.repr_error(Zall, Qb, Rf) <= max(1e-13, 10 * oracle.repr_error(Zall, Qo, Ro))
    assert np.linalg.norm(Rf - Ro) / np.linalg.norm(Ro) <= 1e-10


@pytest.mark.parametrize("variant", VARIANTS)
def test_append_breakdown_column(handle, variant):
    """A zero column in the new block breaks down at that column (1-based
    among the new ones), as in the oracle; the handle stays usable."""
    A, Zall = W.tridiag(2000, 8)
    k = 3
    Qo, Po = oracle_basis(A, Zall[:, :k], variant)
    Z = Zall[:, k:].copy()
    Z[:, 2] = 0.0
    _, _, _, info_o, kind_o, _ = oracle.mgs_append(A, Qo, Po, Z, variant)
    assert (info_o, kind_o) == (3, 1)
    _, _, _, st, info = gpu_append(handle, A, Qo, Po, Z, variant)
    assert (st, info) == (mgsa.MGSA_ERR_BREAKDOWN, 3)
    Q, P, R, st, info = gpu_append(handle, A, Qo, Po, Zall[:, k:], variant)
    assert (st, info) == (mgsa.MGSA_OK, 0)
    check_append(A, Qo, Po, Zall[:, k:], variant, Q, P, R)


def test_append_argument_errors(handle):
    A, Zall = W.tridiag(500, 8)
    Ad = dev_csr(A)
    Qo, Po = (dev_cols(x) for x in oracle_basis(A, Zall[:, :3], "ha"))
    Z = dev_cols(Zall[:, 3:])
    m, n, k = 500, 5, 3
    csr = mgsa.make_csr(m, A[1].size, *Ad)
    Q = torch.empty((n, m), dtype=torch.float64, device="cuda").T
    P = torch.empty((n, m), dtype=torch.float64, device="cuda").T
    R = torch.empty((n, k + n), dtype=torch.float64, device="cuda").T

    def call(**kw):
        a = dict(Qold=Qo, ldqo=m, Pold=Po, ldpo=m, k=k, Z=Z, m=m, n=n, ldz=m, variant=mgsa.MGSA_HA, Q=Q, ldq=m,
                 P=P, ldp=m, R=R, ldr=k + n)
        a.update(kw)
        return mgsa.mgsa_qr_append(handle.h, csr, **a)

    assert call() == mgsa.MGSA_OK
    torch.cuda.synchronize()
    assert call(ldr=k + n - 1) == mgsa.MGSA_ERR_INVALID          # R must hold k + n rows
    assert call(Qold=None) == mgsa.MGSA_ERR_INVALID              # k > 0 needs the given columns
    assert call(Pold=None) == mgsa.MGSA_ERR_INVALID
    assert call(ldqo=m - 1) == mgsa.MGSA_ERR_INVALID
    assert call(k=-1) == mgsa.MGSA_ERR_INVALID
    assert call(k=mgsa.MGSA_MAX_N - n + 1, ldr=mgsa.MGSA_MAX_N + 1) == mgsa.MGSA_ERR_INVALID
    assert call(k=m - n + 1, ldr=m + 1) == mgsa.MGSA_ERR_INVALID  # m < k + n
    assert call(P=Q) == mgsa.MGSA_ERR_INVALID                    # P overlaps Q
    assert call(Q=Qo) == mgsa.MGSA_ERR_INVALID                   # output overlaps a given column
    assert call(P=None) == mgsa.MGSA_OK                          # P is optional
    torch.cuda.synchronize()
    assert handle.info() == (mgsa.MGSA_OK, 0)
