"""Failure detection of the device-wide waits, without a GPU fault.

Every device-wide wait of the whole-GPU MGS kernel is bounded (4 s); when one
runs out the kernel records MGSA_ERR_TIMEOUT in the handle's status word and
every CTA returns.  MGSA_PARAM_WAIT_FAULT starts the barrier counter one
arrival short, so the first wait can never complete: nothing spins forever,
nothing traps, no memory is touched out of bounds.  The tests check that the
host reads the timeout, that the launch ended within the bound, and that the
same handle (and context) then runs a normal QR that matches the oracle.
"""
import time

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402

WAIT_LIMIT_S = 4.0


@pytest.fixture(scope="module")
def handle():
    h = mgsa.Handle(0)
    yield h
    h.close()


def dev(A, Z):
    d = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)
    return Ad, torch.from_numpy(np.ascontiguousarray(np.asarray(Z).T)).to(d).T


def run(h, Ad, Zd, variant):
    Q, R = h.qr(Ad, Zd, variant)
    st = h.info()
    return Q, R, st


@pytest.mark.parametrize("variant,chunk", [("hp", 0), ("naive", 64)])
def test_timeout_is_reported_and_the_handle_recovers(handle, variant, chunk):
    """chunk 0: resident pivots; 64: pivots staged chunk by chunk."""
    A, Z = W.banded(20000, 12, seed=61)
    Ad, Zd = dev(A, Z)
    handle.set_param(mgsa.MGSA_PARAM_CLUSTER, 1)  # the whole-GPU kernel
    handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, chunk)
    try:
        torch.cuda.synchronize()
        handle.set_param(mgsa.MGSA_PARAM_WAIT_FAULT, 1)
        t0 = time.perf_counter()
        try:
            _, _, st = run(handle, Ad, Zd, variant)
        finally:
            handle.set_param(mgsa.MGSA_PARAM_WAIT_FAULT, 0)
        elapsed = time.perf_counter() - t0
        assert st == (mgsa.MGSA_ERR_TIMEOUT, -1)
        assert WAIT_LIMIT_S * 0.9 <= elapsed <= WAIT_LIMIT_S + 20.0, elapsed

        Q, R, st = run(handle, Ad, Zd, variant)
        assert st == (mgsa.MGSA_OK, 0)
        Qo, Ro, info, _, _ = oracle.mgs(A, Z, variant, "row")
        assert info == 0
        Qg, Rg = Q.cpu().numpy(), R.cpu().numpy()
        assert np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro) <= 1e-10
        assert oracle.repr_error(Z, Qg, Rg) <= max(1e-13, 10 * oracle.repr_error(Z, Qo, Ro))
        assert oracle.orth_loss(A, Qg) <= max(1e-12, 10 * oracle.orth_loss(A, Qo))
    finally:
        handle.set_param(mgsa.MGSA_PARAM_CLUSTER, 0)
        handle.set_param(mgsa.MGSA_PARAM_CHUNK_ROWS, 0)


def test_hook_does_not_touch_cluster_launches(handle):
    """A QR small enough for one thread-block cluster uses hardware barriers,
    which the hook leaves alone: it completes normally."""
    A, Z = W.tridiag(1024, 8)
    Ad, Zd = dev(A, Z)
    handle.set_param(mgsa.MGSA_PARAM_WAIT_FAULT, 1)
    try:
        Q, R, st = run(handle, Ad, Zd, "ha")
    finally:
        handle.set_param(mgsa.MGSA_PARAM_WAIT_FAULT, 0)
    assert st == (mgsa.MGSA_OK, 0)
    _, Ro, _, _, _ = oracle.mgs(A, Z, "ha", "row")
    assert np.linalg.norm(R.cpu().numpy() - Ro) / np.linalg.norm(Ro) <= 1e-10


def test_hook_value_range(handle):
    assert mgsa.lib().mgsa_set_param(handle.h, mgsa.MGSA_PARAM_WAIT_FAULT, 2) == mgsa.MGSA_ERR_INVALID
    assert mgsa.lib().mgsa_set_param(handle.h, mgsa.MGSA_PARAM_WAIT_FAULT, 0) == mgsa.MGSA_OK
