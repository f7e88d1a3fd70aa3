"""Grouped launches (mgsa_qr_group): several QRs side by side in one
cooperative launch, each on a gang of CTAs with its own device-wide barrier.

A member's result must equal, bit for bit, that of mgsa_qr on a handle whose
launches use the same plan (MGSA_PARAM_MAX_CTAS = the member's CTAs, no
cluster), whatever else runs in the launch; time slices of a member spread
over several grouped launches must give the same bits as one whole QR; a
member that breaks down reports it in its own status words without touching
the others; gang sizes that change between slices still meet the oracle's
gates; and bad arguments are refused on the host.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402

DEV = torch.device("cuda")


class Member:
    """Device inputs, outputs and workspace of one member."""

    def __init__(self, h, A, Z, variant):
        self.A_host, self.Z_host, self.variant = A, Z, variant
        self.m, self.n = Z.shape
        self.A = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in A)
        self.Z = torch.from_numpy(np.ascontiguousarray(Z.T)).to(DEV).T
        self.Q = torch.empty((self.n, self.m), dtype=torch.float64, device=DEV).T
        self.R = torch.empty((self.n, self.n), dtype=torch.float64, device=DEV).T
        wb = mgsa.mgsa_group_workspace_bytes(h.h, self.m, self.n, mgsa.VARIANTS[variant])
        assert wb > 0
        self.work = torch.empty(wb // 8 + 32, dtype=torch.float64, device=DEV)
        assert self.work.data_ptr() % 256 == 0

    def spec(self, first, count, ctas):
        return mgsa.group_member(self.m, self.n, mgsa.VARIANTS[self.variant], *self.A, self.Z, self.m, self.Q, self.m,
                                 self.R, self.n, self.work, first, count, ctas)

    def status(self):
        return self.work[:1].view(torch.int32)[:2].cpu().tolist()

    def result(self):
        return self.Q.cpu().numpy(), self.R.cpu().numpy()


def reference(A, Z, variant, ctas):
    """mgsa_qr with the plan of a member of `ctas` CTAs."""
    h = mgsa.Handle(0)
    mgsa.mgsa_set_param(h.h, mgsa.MGSA_PARAM_MAX_CTAS, ctas)
    mgsa.mgsa_set_param(h.h, mgsa.MGSA_PARAM_CLUSTER, 1)
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in A)
    Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to(DEV).T
    Q, R = h.qr(Ad, Zd, variant)
    assert h.info() == (mgsa.MGSA_OK, 0)
    out = Q.cpu().numpy(), R.cpu().numpy()
    h.close()
    return out


@pytest.fixture(scope="module")
def handle():
    h = mgsa.Handle(0)
    yield h
    h.close()


@pytest.mark.parametrize("variant", ["naive", "ha", "hp"])
def test_group_members_equal_their_single_launches(handle, variant):
    cases = [(W.banded(20011, 40, seed=31), 40), (W.poisson2d(side=150, n=24), 24), (W.tridiag(5003, 7), 7),
             (W.varcoef3d(side=24, n=16), 60)]
    members = [Member(handle, A, Z, variant) for (A, Z), _ in cases]
    specs = [mb.spec(0, mb.n, ctas) for mb, (_, ctas) in zip(members, cases)]
    assert mgsa.mgsa_qr_group(handle.h, mgsa.VARIANTS[variant], specs) == mgsa.MGSA_OK, mgsa.mgsa_last_error()
    torch.cuda.synchronize()
    for mb, ((A, Z), ctas) in zip(members, cases):
        assert mb.status() == [0, 0]
        Q, R = mb.result()
        Qr, Rr = reference(A, Z, variant, ctas)
        assert np.array_equal(R, Rr) and np.array_equal(Q, Qr), (variant, mb.m, ctas)


def test_group_time_slices_equal_one_qr(handle):
    """Member 0 runs in three slices, next to different companions each time."""
    A0, Z0 = W.banded(30011, 33, seed=32)
    big = Member(handle, A0, Z0, "hp")
    others = [Member(handle, *W.tridiag(4000 + 1000 * k, 6 + k), "hp") for k in range(3)]
    for (first, count), other in zip([(0, 10), (10, 5), (15, 18)], others):
        specs = [big.spec(first, count, 48), other.spec(0, other.n, 20)]
        assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_HP, specs) == mgsa.MGSA_OK, mgsa.mgsa_last_error()
    torch.cuda.synchronize()
    assert big.status() == [0, 0]
    Q, R = big.result()
    Qr, Rr = reference(A0, Z0, "hp", 48)
    assert np.array_equal(R, Rr) and np.array_equal(Q, Qr)
    for other in others:
        assert other.status() == [0, 0]


def test_group_gang_size_changing_between_slices_meets_oracle_gates(handle):
    A, Z = W.varcoef3d(side=26, n=20)
    mb = Member(handle, A, Z, "ha")
    for first, count, ctas in [(0, 7, 100), (7, 6, 13), (13, 7, 57)]:
        assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_HA, [mb.spec(first, count, ctas)]) == mgsa.MGSA_OK
    torch.cuda.synchronize()
    assert mb.status() == [0, 0]
    Q, R = mb.result()
    Qo, Ro, info, _, _ = oracle.mgs(A, Z, "ha", "row")
    assert info == 0
    assert oracle.repr_error(Z, Q, R) <= max(1e-13, 10 * oracle.repr_error(Z, Qo, Ro))
    assert oracle.orth_loss(A, Q) <= max(1e-12, 10 * oracle.orth_loss(A, Qo))
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10
    kR = np.linalg.cond(Ro)
    assert np.abs(Q - Qo).max() <= 1e-9 * kR * np.abs(Qo).max()


def test_group_breakdown_stays_in_its_member(handle):
    A, Z = W.tridiag(3000, 6)
    Zb = np.asfortranarray(Z.copy())
    Zb[:, 4] = 0.0
    bad = Member(handle, A, Zb, "hp")
    good = Member(handle, *W.banded(9000, 12, seed=33), "hp")
    # two slices: the one after the failure must do nothing to `bad`
    for first, count in [(0, 5), (5, 1)]:
        specs = [bad.spec(first, count, 10), good.spec(0 if first == 0 else 0, good.n, 30)]
        assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_HP, specs) == mgsa.MGSA_OK
    torch.cuda.synchronize()
    assert bad.status() == [mgsa.MGSA_ERR_BREAKDOWN, 5]
    assert good.status() == [0, 0]
    Q, R = good.result()
    Qr, Rr = reference(good.A_host, good.Z_host, "hp", 30)
    assert np.array_equal(R, Rr) and np.array_equal(Q, Qr)


def test_group_argument_errors(handle):
    mb = Member(handle, *W.tridiag(2000, 5), "hp")
    big = [Member(handle, *W.tridiag(40000, 5), "hp") for _ in range(2)]
    sms = torch.cuda.get_device_properties(DEV).multi_processor_count
    too_many = [big[0].spec(0, 5, sms), big[1].spec(0, 5, sms)]  # 40000 rows take 152 slabs of 128+ rows each
    assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_HP, too_many) == mgsa.MGSA_ERR_INVALID
    assert "CTAs" in mgsa.mgsa_last_error()
    shared = [mb.spec(0, 5, 4), mb.spec(0, 5, 4)]  # two members on one workspace
    assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_HP, shared) == mgsa.MGSA_ERR_INVALID
    assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_HA, [mb.spec(0, 5, 4)]) == mgsa.MGSA_ERR_INVALID  # variant
    assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_HP, [mb.spec(3, 3, 4)]) == mgsa.MGSA_ERR_INVALID  # past n
    assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_HP, [mb.spec(0, 5, 0)]) == mgsa.MGSA_ERR_INVALID  # ctas
    assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_CGS_HP, [mb.spec(0, 5, 4)]) == mgsa.MGSA_ERR_INVALID
    spec = mb.spec(0, 5, 4)
    spec.job.work += 8  # misaligned workspace
    assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_HP, [spec]) == mgsa.MGSA_ERR_INVALID
    assert mgsa.mgsa_qr_group(handle.h, mgsa.MGSA_HP, []) == mgsa.MGSA_ERR_INVALID
