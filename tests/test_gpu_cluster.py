"""Small QRs on one thread-block cluster (hardware cluster barriers instead of
the device-wide ones): parity with the oracle for every MGS form, automatic
and forced cluster sizes, long rows, the successive orthogonalisation;
deterministic; the same factors as the whole-GPU launch to rounding."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402

FORMS = ["naive", "ha", "hp"]


@pytest.fixture(scope="module")
def handle():
    h = mgsa.Handle(0)
    yield h
    h.close()


def dev(A, Z):
    d = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)
    return Ad, torch.from_numpy(np.ascontiguousarray(np.asarray(Z).T)).to(d).T


def qr(h, A, Z, variant, cluster):
    h.set_param(mgsa.MGSA_PARAM_CLUSTER, cluster)
    try:
        Ad, Zd = dev(A, Z)
        Q, R = h.qr(Ad, Zd, variant)
        return Q.cpu().numpy(), R.cpu().numpy(), h.info()
    finally:
        h.set_param(mgsa.MGSA_PARAM_CLUSTER, 0)


def check(A, Z, variant, Q, R):
    Qo, Ro, info, _, _ = oracle.mgs(A, Z, variant, "row")
    assert info == 0
    assert oracle.repr_error(Z, Q, R) <= max(1e-13, 10 * oracle.repr_error(Z, Qo, Ro))
    assert oracle.orth_loss(A, Q) <= max(1e-12, 10 * oracle.orth_loss(A, Qo))
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10


CASES = {
    "tridiag_1x1": lambda: W.tridiag(1, 1),
    "tridiag_17x3": lambda: W.tridiag(17, 3),
    "tridiag_4096x16": lambda: W.tridiag(4096, 16),
    "tridiag_5003x7": lambda: W.tridiag(5003, 7),
    "banded_3000x64": lambda: W.banded(3000, 64, seed=4),
    "denseband_2000x24": lambda: W.denseband(2000, 24, hb=100),
    "banded_40000x12": lambda: W.banded(40000, 12, seed=44),  # 2500 rows per CTA of 16
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("variant", FORMS)
@pytest.mark.parametrize("cluster", [0, 2, 8])
def test_cluster_parity(handle, case, variant, cluster):
    A, Z = CASES[case]()
    Q, R, info = qr(handle, A, Z, variant, cluster)
    assert info == (mgsa.MGSA_OK, 0)
    check(A, Z, variant, Q, R)


@pytest.mark.parametrize("variant", FORMS)
def test_largest_cluster_and_grid_agree(handle, variant):
    """A 16-CTA cluster needs the non-portable size; where the GPU cannot
    co-schedule it the call is refused with MGSA_ERR_INVALID, never run on
    fewer CTAs than asked.  The first size that launches matches the oracle
    and the whole-GPU launch to rounding."""
    A, Z = W.tridiag(4096, 16)
    Ad, Zd = dev(A, Z)
    m, n = Z.shape
    csr = mgsa.make_csr(m, Ad[1].numel(), *Ad)
    Q = torch.empty((n, m), dtype=torch.float64, device="cuda").T
    R = torch.empty((n, n), dtype=torch.float64, device="cuda").T
    for c in (16, 12, 8):
        handle.set_param(mgsa.MGSA_PARAM_CLUSTER, c)
        try:
            st = mgsa.mgsa_qr(handle.h, csr, Zd, m, n, m, mgsa.VARIANTS[variant], Q, m, R, n)
        finally:
            handle.set_param(mgsa.MGSA_PARAM_CLUSTER, 0)
        if st == mgsa.MGSA_OK:
            break
        assert st == mgsa.MGSA_ERR_INVALID
    else:
        pytest.fail("no cluster of 8..16 CTAs could be launched")
    assert handle.info() == (mgsa.MGSA_OK, 0)
    Qc, Rc = Q.cpu().numpy(), R.cpu().numpy()
    check(A, Z, variant, Qc, Rc)
    Qg, Rg, info = qr(handle, A, Z, variant, 1)
    assert info == (mgsa.MGSA_OK, 0)
    assert np.linalg.norm(Rc - Rg) / np.linalg.norm(Rg) <= 1e-13
    assert np.abs(Qc - Qg).max() <= 1e-12 * np.abs(Qg).max()


@pytest.mark.parametrize("variant", FORMS)
def test_cluster_deterministic(handle, variant):
    A, Z = W.banded(20000, 20, seed=45)
    Q1, R1, i1 = qr(handle, A, Z, variant, 8)
    Q2, R2, i2 = qr(handle, A, Z, variant, 8)
    assert i1 == i2 == (mgsa.MGSA_OK, 0)
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2)


@pytest.mark.parametrize("variant", FORMS)
def test_cluster_breakdown(handle, variant):
    A, Z = W.tridiag(3000, 6)
    Z = Z.copy()
    Z[:, 4] = 0.0
    _, _, info = qr(handle, A, Z, variant, 4)
    assert info == (mgsa.MGSA_ERR_BREAKDOWN, 5)
    A2, Z2 = W.tridiag(3000, 6)
    Q, R, info = qr(handle, A2, Z2, variant, 4)
    assert info == (mgsa.MGSA_OK, 0)
    check(A2, Z2, variant, Q, R)


@pytest.mark.parametrize("variant", FORMS)
def test_append_on_a_cluster(handle, variant):
    A, Zall = W.banded(8000, 20, seed=46)
    k = 6
    Qo, Po, _, info, _, _ = oracle.mgs_append(A, None, None, Zall[:, :k], variant)
    assert info == 0
    handle.set_param(mgsa.MGSA_PARAM_CLUSTER, 4)
    try:
        Ad, _ = dev(A, Zall)
        Q, P, R = handle.append(Ad, dev(A, Qo)[1], dev(A, Po)[1], dev(A, Zall[:, k:])[1], variant)
        assert handle.info() == (mgsa.MGSA_OK, 0)
    finally:
        handle.set_param(mgsa.MGSA_PARAM_CLUSTER, 0)
    Qr, Pr, Rr, info, _, _ = oracle.mgs_append(A, Qo, Po, Zall[:, k:], variant)
    assert info == 0
    assert np.linalg.norm(R.cpu().numpy() - Rr) / np.linalg.norm(Rr) <= 1e-10


def test_cluster_parameter_range(handle):
    assert mgsa.lib().mgsa_set_param(handle.h, mgsa.MGSA_PARAM_CLUSTER, 17) == mgsa.MGSA_ERR_INVALID
    assert mgsa.lib().mgsa_set_param(handle.h, mgsa.MGSA_PARAM_CLUSTER, 0) == mgsa.MGSA_OK
