"""mgsa_qr_noalloc, the allocation-free entry point, against mgsa_qr and the oracle.

mgsa_qr_noalloc is for callers that must not allocate device memory -- code
under a memory manager that owns the whole GPU, or a latency-critical loop
that cannot pay for cudaMalloc's device-wide synchronisation.  Its scratch is
one static device array inside the library, shared by every call.  It runs
the same kernel as mgsa_qr with the same launch plan (whole GPU, no cluster),
so the two must agree bit for bit; each result is also held to the oracle's
gates directly.  Calls run back to back (different sizes and forms, so each
runs on what the previous one left in the array), one runs in place
(Q == Z), and a plain-C client checks that a call after cudaDeviceReset in
its own process redoes the per-context set-up and gives the same bits.  This
file is named so that pytest collects it last.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402

CASES = [("hp", lambda: W.banded(5003, 24, seed=21)), ("ha", lambda: W.poisson2d(side=96, n=32)),
         ("naive", lambda: W.varcoef3d(side=20, n=16))]


def _dev(A, Z):
    d = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)
    Zd = torch.from_numpy(np.ascontiguousarray(np.asarray(Z).T)).to(d).T
    return Ad, Zd


def _noalloc(Ad, Zd, variant, in_place=False):
    m, n = Zd.shape
    Q = Zd if in_place else torch.empty((n, m), dtype=torch.float64, device="cuda").T
    R = torch.empty((n, n), dtype=torch.float64, device="cuda").T
    info = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    csr = mgsa.make_csr(m, Ad[1].numel(), *Ad)
    st = mgsa.mgsa_qr_noalloc(csr, Zd, m, n, m, mgsa.VARIANTS[variant], Q, m, R, n, info)
    return st, (Q, R, info)


def _oracle_gates(A, Z, variant, Q, R):
    """The parity gates of the other GPU tests, against the same form of the oracle."""
    Qo, Ro, info, _, _ = oracle.mgs(A, Z, variant, "row")
    assert info == 0
    assert oracle.repr_error(Z, Q, R) <= max(1e-13, 10 * oracle.repr_error(Z, Qo, Ro))
    assert oracle.orth_loss(A, Q) <= max(1e-12, 10 * oracle.orth_loss(A, Qo))
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10
    kR = np.linalg.cond(Ro)
    assert np.abs(R - Ro).max() <= 1e-9 * kR * np.abs(Ro).max()
    assert np.abs(Q - Qo).max() <= 1e-9 * kR * np.abs(Qo).max()


@pytest.fixture(scope="module")
def whole_gpu_handle():
    h = mgsa.Handle(0)
    mgsa.mgsa_set_param(h.h, mgsa.MGSA_PARAM_CLUSTER, 1)  # the plan mgsa_qr_noalloc uses
    yield h
    h.close()


def test_noalloc_matches_mgsa_qr_on_calls_in_a_row(whole_gpu_handle):
    assert torch.cuda.is_available()
    inputs = [(v, *gen()) for v, gen in CASES]
    # Allocation-free calls back to back on the same stream, every form.
    runs = []
    for variant, A, Z in inputs:
        Ad, Zd = _dev(A, Z)
        st, out = _noalloc(Ad, Zd, variant)
        assert st == mgsa.MGSA_OK, mgsa.mgsa_last_error()
        runs.append((Ad, Zd, *out))
    torch.cuda.synchronize()
    # The same inputs through the allocating entry point: the same bits.
    h = whole_gpu_handle
    for (variant, A, Z), (Ad, Zd, Q, R, info) in zip(inputs, runs):
        assert info.cpu().tolist() == [0, 0]
        Qr, Rr = h.qr(Ad, Zd, variant)
        assert h.info() == (mgsa.MGSA_OK, 0)
        Qn, Rn = Q.cpu().numpy(), R.cpu().numpy()
        assert np.array_equal(Rn, Rr.cpu().numpy()), variant
        assert np.array_equal(Qn, Qr.cpu().numpy()), variant
        _oracle_gates(A, Z, variant, Qn, Rn)


def test_noalloc_in_place_equals_separate_q(whole_gpu_handle):
    A, Z = W.banded(4099, 20, seed=22)
    for variant in ("hp", "naive"):
        Ad, Zd = _dev(A, Z)
        Qr, Rr = whole_gpu_handle.qr(Ad, Zd, variant)
        assert whole_gpu_handle.info() == (mgsa.MGSA_OK, 0)
        st, (Q, R, info) = _noalloc(Ad, Zd, variant, in_place=True)
        assert st == mgsa.MGSA_OK, mgsa.mgsa_last_error()
        assert Q.data_ptr() == Zd.data_ptr()
        assert info.cpu().tolist() == [0, 0]
        assert np.array_equal(R.cpu().numpy(), Rr.cpu().numpy()), variant
        assert np.array_equal(Q.cpu().numpy(), Qr.cpu().numpy()), variant


def test_noalloc_reports_breakdown_in_info_dev():
    A, Z = W.tridiag(600, 6)
    Z = np.asfortranarray(Z.copy())
    Z[:, 3] = 0.0
    Ad, Zd = _dev(A, Z)
    st, (_, _, info) = _noalloc(Ad, Zd, "hp")
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


@pytest.mark.parametrize("variant", [0, 2])
def test_noalloc_after_device_reset_in_a_c_client(tmp_path, variant):
    from c_client import build_client

    exe = build_client(str(tmp_path), "noalloc_reset")
    r = subprocess.run([exe, "3000", "8", str(variant)], capture_output=True, text=True, timeout=120,
                       env={**os.environ, "CUDA_VISIBLE_DEVICES": os.environ.get("CUDA_VISIBLE_DEVICES", "0")})
    assert r.returncode == 0 and r.stdout.startswith("ok"), (r.stdout, r.stderr)
