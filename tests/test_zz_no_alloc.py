"""mgsa_qr_noalloc, the allocation-free entry point, against mgsa_qr.

mgsa_qr_noalloc is for callers that must not allocate device memory -- code
under a memory manager that owns the whole GPU, or a latency-critical loop
that cannot pay for cudaMalloc's device-wide synchronisation.  Its scratch is
one static device array inside the library, shared by every call.  Here two
calls in a row (different sizes and variants, so the second runs on what the
first left in the array) are each checked, through the C-ABI, against the
allocating entry point mgsa_qr on the same input, within the parity tolerance
the other GPU tests use.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402


def _dev(A, Z):
    d = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)
    Zd = torch.from_numpy(np.ascontiguousarray(np.asarray(Z).T)).to(d).T
    return Ad, Zd


def _noalloc(A, Z, variant):
    Ad, Zd = _dev(A, Z)
    m, n = Zd.shape
    Q = torch.empty((n, m), dtype=torch.float64, device="cuda").T
    R = torch.empty((n, n), dtype=torch.float64, device="cuda").T
    info = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    csr = mgsa.make_csr(m, Ad[1].numel(), *Ad)
    st = mgsa.mgsa_qr_noalloc(csr, Zd, m, n, m, mgsa.VARIANTS[variant], Q, m, R, n, info)
    return st, (Ad, Zd, Q, R, info)


def _close(Q, R, Qr, Rr):
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= 1e-10
    kR = np.linalg.cond(Rr)
    assert np.abs(R - Rr).max() <= 1e-9 * kR * np.abs(Rr).max()
    assert np.abs(Q - Qr).max() <= 1e-9 * kR * np.abs(Qr).max()


def test_noalloc_matches_mgsa_qr_on_two_calls_in_a_row():
    assert torch.cuda.is_available()
    cases = [("hp", W.banded(5003, 24, seed=21)), ("ha", W.poisson2d(side=96, n=32))]
    # Two allocation-free calls back to back on the same stream.
    runs = []
    for variant, (A, Z) in cases:
        st, bufs = _noalloc(A, Z, variant)
        assert st == mgsa.MGSA_OK, mgsa.mgsa_last_error()
        runs.append(bufs)
    torch.cuda.synchronize()
    # The same inputs through the allocating entry point.
    with mgsa.Handle(0) as h:
        for (variant, (A, Z)), (Ad, Zd, Q, R, info) in zip(cases, runs):
            assert info.cpu().tolist() == [0, 0]
            Qr, Rr = h.qr(Ad, Zd, variant)
            assert h.info() == (mgsa.MGSA_OK, 0)
            _close(Q.cpu().numpy(), R.cpu().numpy(), Qr.cpu().numpy(), Rr.cpu().numpy())


def test_noalloc_reports_breakdown_in_info_dev():
    A, Z = W.tridiag(600, 6)
    Z = np.asfortranarray(Z.copy())
    Z[:, 3] = 0.0
    st, (_, _, _, _, info) = _noalloc(A, Z, "hp")
    assert st == mgsa.MGSA_OK
    assert info.cpu().tolist() == [mgsa.MGSA_ERR_BREAKDOWN, 4]


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    m, n = 262144, 32  # HP needs m * n * 8 = 64 MiB of x columns > 32 MiB
    A = W.tridiag_csr(m)
    Ad, _ = _dev(A, np.zeros((1, 1)))
    Z = torch.zeros((n, m), dtype=torch.float64, device="cuda").T
    Q = torch.empty((n, m), dtype=torch.float64, device="cuda").T
    R = torch.empty((n, n), dtype=torch.float64, device="cuda").T
    csr = mgsa.make_csr(m, Ad[1].numel(), *Ad)
    st = mgsa.mgsa_qr_noalloc(csr, Z, m, n, m, mgsa.MGSA_HP, Q, m, R, n, None)
    assert st == mgsa.MGSA_ERR_INVALID
    assert "MGSA_NOALLOC_SCRATCH_BYTES" in mgsa.mgsa_last_error()
