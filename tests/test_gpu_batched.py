"""mgsa_qr_batched: many independent instances in one call, through the C-ABI.

Every job is checked against the CPU oracle with the gates of
test_gpu_parity.py and against the single-instance entry point mgsa_qr
(same algorithm, different reduction tree: agreement within tolerance).
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402
from paper_1703_10440_gb300.batch import Batch  # noqa: E402

VARIANTS = ["naive", "ha", "hp"]


@pytest.fixture(scope="module")
def handle():
    h = mgsa.Handle(0)
    yield h
    h.close()


def mixed_instances(count, seed=11, m_hi=6000, n_hi=64):
    g = W.rng(seed, 300)
    out = []
    for k in range(count):
        n = int(g.integers(1, n_hi + 1))
        m = int(max(n, np.rint(np.exp(g.uniform(np.log(max(n, 2)), np.log(m_hi))))))
        kind = k % 3
        if kind == 0:
            A, Z = W.banded(m, n, seed=seed, index=k)
        elif kind == 1:
            A, Z = W.tridiag(m, n, seed=seed + k)
        else:
            side = int(max(2, np.sqrt(m)))
            A = W.laplace2d_csr(side, side, 0.05)
            Z = W.gaussian_Z(side * side, min(n, side * side), seed + k)
        out.append((A, Z))
    out.append(W.tridiag(1, 1))       # m = n = 1
    out.append(W.banded(40, 40, seed=3))  # m = n
    out.append(W.banded(4096, 17, seed=4))  # largest resident slab
    out.append(W.banded(8200, 9, seed=5))   # two chunks
    out.append(W.denseband(1500, 20, hb=60))  # long rows: warp-per-row MVs
    out.append(W.denseband(6000, 12, hb=40))  # long rows, two chunks
    return out


def gates(A, Z, variant, Q, R):
    Qo, Ro, info, _, _ = oracle.mgs(A, Z, variant, "row")
    assert info == 0
    assert oracle.repr_error(Z, Q, R) <= max(1e-13, 10 * oracle.repr_error(Z, Qo, Ro))
    assert oracle.orth_loss(A, Q) <= max(1e-12, 10 * oracle.orth_loss(A, Qo))
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) > 0)
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10


def test_batched_matches_oracle_and_single(handle):
    inst = mixed_instances(36)
    variants = [VARIANTS[k % 3] for k in range(len(inst))]
    b = Batch(inst, variants)
    b.run(handle.h)
    torch.cuda.synchronize()
    assert np.all(b.infos() == 0), b.infos()
    for k, ((A, Z), v) in enumerate(zip(inst, variants)):
        Q, R, info = b.result(k)
        gates(A, Z, v, Q, R)
        d = torch.device("cuda")
        Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)
        Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to(d).T
        Qs, Rs = handle.qr(Ad, Zd, v)
        assert handle.info() == (0, 0)
        Rs = Rs.cpu().numpy()
        assert np.linalg.norm(R - Rs) / np.linalg.norm(Rs) <= 1e-12
        assert np.abs(Q - Qs.cpu().numpy()).max() <= 1e-10 * np.abs(Q).max() * np.linalg.cond(Rs)


def test_batched_deterministic(handle):
    inst = mixed_instances(20, seed=12)
    b = Batch(inst, "hp")
    b.run(handle.h)
    first = [b.result(k) for k in range(b.count)]
    b.Q.zero_()
    b.R.zero_()
    b.run(handle.h)
    for k in range(b.count):
        Q, R, _ = b.result(k)
        assert np.array_equal(Q, first[k][0]) and np.array_equal(R, first[k][1])


def test_batched_reports_bad_jobs_without_touching_others(handle):
    good = W.banded(500, 10, seed=13)
    zero_col = W.banded(300, 6, seed=14)
    zero_col = (zero_col[0], np.asfortranarray(zero_col[1].copy()))
    zero_col[1][:, 3] = 0.0
    nan = W.tridiag(200, 5)
    nan = (nan[0], np.asfortranarray(nan[1].copy()))
    nan[1][7, 2] = np.nan
    too_wide = W.tridiag(400, mgsa.MGSA_BATCH_MAX_N + 1)
    b = Batch([good, zero_col, nan, too_wide, good], ["ha", "hp", "naive", "hp", 7])
    b.run(handle.h)
    torch.cuda.synchronize()
    info = b.infos()
    assert info[0] == 0
    assert info[1] == 4
    assert info[2] == -3
    assert info[3] == mgsa.MGSA_BATCH_INFO_INVALID
    assert info[4] == mgsa.MGSA_BATCH_INFO_INVALID
    Q, R, _ = b.result(0)
    gates(*good, "ha", Q, R)


def test_batched_empty_and_invalid_arguments(handle):
    assert mgsa.mgsa_qr_batched(handle.h, 0, None, None) == mgsa.MGSA_OK
    assert mgsa.mgsa_qr_batched(handle.h, -1, None, None) == mgsa.MGSA_ERR_INVALID
    assert mgsa.mgsa_qr_batched(handle.h, 3, None, None) == mgsa.MGSA_ERR_INVALID
    assert mgsa.mgsa_qr_batched(0, 1, None, None) == mgsa.MGSA_ERR_INVALID


def test_batched_cuda_graph_capture(handle):
    inst = mixed_instances(12, seed=15)
    b = Batch(inst, [VARIANTS[k % 3] for k in range(len(inst))])
    b.run(handle.h)
    torch.cuda.synchronize()
    eager = [b.result(k) for k in range(b.count)]
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    b.Q.zero_()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        b.run(handle.h, s)
    for _ in range(2):
        b.Q.zero_()
        b.R.zero_()
        g.replay()
        torch.cuda.synchronize()
        for k in range(b.count):
            Q, R, info = b.result(k)
            assert info == 0
            assert np.array_equal(Q, eager[k][0]) and np.array_equal(R, eager[k][1])
