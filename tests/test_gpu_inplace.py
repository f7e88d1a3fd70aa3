"""In-place factorisation (Q is Z itself): the same results, bit for bit, as
with a separate Q, for every form, in resident and staged launches, for the
successive orthogonalisation too; any other overlap of Q and Z is refused."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402

FORMS = ["naive", "ha", "hp", "cgs_naive", "cgs_ha", "cgs_hp"]


@pytest.fixture(scope="module")
def handle():
    h = mgsa.Handle(0)
    yield h
    h.close()


def dev(A, Z):
    d = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)
    return Ad, torch.from_numpy(np.ascontiguousarray(np.asarray(Z).T)).to(d).T


def qr_in_place(h, Ad, Zd, variant):
    m, n = Zd.shape
    Zw = Zd.T.clone().T  # a column-major copy that becomes Q
    R = torch.empty((n, n), dtype=torch.float64, device=Zd.device).T
    csr = mgsa.make_csr(m, Ad[1].numel(), *Ad)
    st = mgsa.mgsa_qr(h.h, csr, Zw, m, n, Zw.stride(1), mgsa.VARIANTS[variant], Zw, Zw.stride(1), R, R.stride(1))
    assert st == mgsa.MGSA_OK
    assert h.info() == (mgsa.MGSA_OK, 0)
    return Zw, R


@pytest.mark.parametrize("variant", FORMS)
@pytest.mark.parametrize("staged", [False, True])
def test_in_place_equals_separate(handle, variant, staged):
    A, Z = W.banded(20011, 24, seed=21)
    Ad, Zd = dev(A, Z)
    if staged:
        handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, 3)
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 1024)
    try:
        Q, R = handle.qr(Ad, Zd, variant)
        assert handle.info() == (mgsa.MGSA_OK, 0)
        Qi, Ri = qr_in_place(handle, Ad, Zd, variant)
    finally:
        handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, 0)
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 0)
    assert torch.equal(Q, Qi) and torch.equal(R, Ri)


@pytest.mark.parametrize("variant", ["ha", "hp"])
def test_in_place_long_rows(handle, variant):
    A, Z = W.denseband(2000, 24, hb=100)
    Ad, Zd = dev(A, Z)
    Q, R = handle.qr(Ad, Zd, variant)
    Qi, Ri = qr_in_place(handle, Ad, Zd, variant)
    assert torch.equal(Q, Qi) and torch.equal(R, Ri)


@pytest.mark.parametrize("variant", ["naive", "ha", "hp"])
def test_append_in_place(handle, variant):
    A, Zall = W.banded(9001, 20, seed=22)
    Ad, Zd = dev(A, Zall)
    k = 8
    Q1, P1, _ = handle.append(Ad, None, None, Zd[:, :k], variant)
    Z2 = Zd[:, k:].T.clone().T
    Q2, P2, R2 = handle.append(Ad, Q1, P1, Z2, variant)
    m, n = Z2.shape
    Zw = Z2.T.clone().T
    P = torch.empty((n, m), dtype=torch.float64, device=Zw.device).T
    R = torch.empty((n, k + n), dtype=torch.float64, device=Zw.device).T
    csr = mgsa.make_csr(m, Ad[1].numel(), *Ad)
    st = mgsa.mgsa_qr_append(handle.h, csr, Q1, Q1.stride(1), P1, P1.stride(1), k, Zw, m, n, Zw.stride(1),
                             mgsa.VARIANTS[variant], Zw, Zw.stride(1), P, P.stride(1), R, R.stride(1))
    assert st == mgsa.MGSA_OK and handle.info() == (mgsa.MGSA_OK, 0)
    assert torch.equal(Zw, Q2) and torch.equal(P, P2) and torch.equal(R, R2)


def test_partial_overlap_refused(handle):
    A, Z = W.tridiag(500, 4)
    Ad, Zd = dev(A, Z)
    m, n = Zd.shape
    buf = torch.zeros((n + 1) * m, dtype=torch.float64, device="cuda")
    Zw = buf[: n * m].view(n, m).T
    Zw.copy_(Zd)
    Qs = buf[m // 2: m // 2 + n * m].view(n, m).T  # shifted by half a column
    R = torch.empty((n, n), dtype=torch.float64, device="cuda").T
    csr = mgsa.make_csr(m, Ad[1].numel(), *Ad)
    assert mgsa.mgsa_qr(handle.h, csr, Zw, m, n, m, mgsa.MGSA_HA, Qs, m, R, n) == mgsa.MGSA_ERR_INVALID
    # the same pointer with another leading dimension is an overlap too
    big = torch.zeros(n * (m + 8), dtype=torch.float64, device="cuda")
    Zb = big.view(n, m + 8).T[:m]
    assert mgsa.mgsa_qr(handle.h, csr, Zb, m, n, m + 8, mgsa.MGSA_HA, Zb, m, R, n) == mgsa.MGSA_ERR_INVALID
