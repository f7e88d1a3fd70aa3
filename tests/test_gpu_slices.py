"""Time-sliced QR (mgsa_qr_steps): the slices of one QR, run in order, give
bit for bit the results of one mgsa_qr call -- for every MGS form, resident
and staged launches, long rows, any slice length -- also with other work on
another handle between the slices; a failure in one slice stops the rest."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402

FORMS = ["naive", "ha", "hp"]


@pytest.fixture(scope="module")
def handle():
    # Slices always run on the whole GPU; the one-call reference must too.
    h = mgsa.Handle(0)
    h.set_param(mgsa.MGSA_PARAM_CLUSTER, 1)
    yield h
    h.close()


def dev(A, Z):
    d = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)
    return Ad, torch.from_numpy(np.ascontiguousarray(np.asarray(Z).T)).to(d).T


def sliced(h, Ad, Zd, variant, count, between=None):
    m, n = Zd.shape
    Q = torch.empty((n, m), dtype=torch.float64, device=Zd.device).T
    R = torch.full((n, n), 7.0, dtype=torch.float64, device=Zd.device).T
    csr = mgsa.make_csr(m, Ad[1].numel(), *Ad)
    for first in range(0, n, count):
        st = mgsa.mgsa_qr_steps(h.h, csr, Zd, m, n, Zd.stride(1), mgsa.VARIANTS[variant], Q, m, R, n, first,
                                min(count, n - first))
        assert st == mgsa.MGSA_OK, mgsa.mgsa_last_error()
        if between is not None:
            between()
    return Q, R, h.info()


CASES = {
    "banded_20011x24": (lambda: W.banded(20011, 24, seed=41), None),
    "tridiag_257x33": (lambda: W.tridiag(257, 33), None),
    "denseband_2000x24": (lambda: W.denseband(2000, 24, hb=100), None),
    "banded_5003x12_staged": (lambda: W.banded(5003, 12, seed=6), (3, 1024)),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("variant", FORMS)
@pytest.mark.parametrize("count", [1, 5, 8])
def test_slices_equal_one_call(handle, case, variant, count):
    gen, tiling = CASES[case]
    A, Z = gen()
    Ad, Zd = dev(A, Z)
    if tiling:
        handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, tiling[0])
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, tiling[1])
    try:
        Q1, R1 = handle.qr(Ad, Zd, variant)
        assert handle.info() == (mgsa.MGSA_OK, 0)
        Q2, R2, info = sliced(handle, Ad, Zd, variant, count)
    finally:
        handle.set_param(mgsa.MGSA_PARAM_MAX_CTAS, 0)
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 0)
    assert info == (mgsa.MGSA_OK, 0)
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)


@pytest.mark.parametrize("variant", FORMS)
def test_other_work_between_slices(handle, variant):
    A, Z = W.banded(30011, 20, seed=42)
    Ad, Zd = dev(A, Z)
    Q1, R1 = handle.qr(Ad, Zd, variant)
    assert handle.info() == (mgsa.MGSA_OK, 0)
    other = mgsa.Handle(0)
    B, Y = W.tridiag(4000, 9)
    Bd, Yd = dev(B, Y)
    results = []

    def between():
        results.append(other.qr(Bd, Yd, "hp"))

    try:
        Q2, R2, info = sliced(handle, Ad, Zd, variant, 3, between)
        assert other.info() == (mgsa.MGSA_OK, 0)
    finally:
        other.close()
    assert info == (mgsa.MGSA_OK, 0)
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)
    for Qo, Ro in results[1:]:
        assert torch.equal(Qo, results[0][0]) and torch.equal(Ro, results[0][1])


@pytest.mark.parametrize("variant", FORMS)
def test_failure_stops_later_slices(handle, variant):
    A, Z = W.banded(9001, 16, seed=43)
    Z = Z.copy()
    Z[:, 7] = 0.0  # breakdown at column 8
    Ad, Zd = dev(A, Z)
    handle.qr(Ad, Zd, variant)
    expect = handle.info()
    assert expect == (mgsa.MGSA_ERR_BREAKDOWN, 8)
    _, _, info = sliced(handle, Ad, Zd, variant, 3)
    assert info == expect
    # the handle is usable afterwards
    A2, Z2 = W.tridiag(3000, 5)
    Ad2, Zd2 = dev(A2, Z2)
    handle.qr(Ad2, Zd2, variant)
    assert handle.info() == (mgsa.MGSA_OK, 0)


def test_slice_arguments(handle):
    A, Z = W.tridiag(500, 6)
    Ad, Zd = dev(A, Z)
    m, n = Zd.shape
    Q = torch.empty((n, m), dtype=torch.float64, device="cuda").T
    R = torch.empty((n, n), dtype=torch.float64, device="cuda").T
    csr = mgsa.make_csr(m, Ad[1].numel(), *Ad)

    def call(first, count, v=mgsa.MGSA_HA):
        return mgsa.mgsa_qr_steps(handle.h, csr, Zd, m, n, m, v, Q, m, R, n, first, count)

    assert call(0, 0) == mgsa.MGSA_ERR_INVALID
    assert call(-1, 2) == mgsa.MGSA_ERR_INVALID
    assert call(6, 1) == mgsa.MGSA_ERR_INVALID
    assert call(4, 3) == mgsa.MGSA_ERR_INVALID
    assert call(0, 6, mgsa.MGSA_CGS_HA) == mgsa.MGSA_ERR_INVALID
    assert call(0, 6) == mgsa.MGSA_OK
    assert handle.info() == (mgsa.MGSA_OK, 0)
