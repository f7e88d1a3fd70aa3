"""Parity at the full workload sizes, in the launch configuration bench.py uses.

Each form (naive, HA, HP) is compared with the same form of the oracle on the
same input, element by element over all of Q and R.  The oracle here is its
multi-core build (``oracle.mgs_par``), which performs the single-thread
oracle's operations in the same order and returns the same bits (pinned by
``test_oracle_par.py``); it finishes a 128^3 QR in seconds on the host's cores.

Gates (as in ``test_gpu_parity.py``, from Section 3's error analysis):
  ||R - R_oracle||_F / ||R||_F <= 1e-10 where kappa(Z) <= 1e3;
  |Q - Q_oracle| <= 1e-9 kappa(R) max|Q_oracle|, likewise R;
  ||Z - QR||_F / ||Z||_F <= max(1e-13, 10 x oracle's),
  ||I - Q^T A Q||_F <= max(1e-12, 10 x oracle's).
The two norms are evaluated on the GPU in FP64 with torch (test
infrastructure), for the CUDA result and for the oracle's.  Properties that
hold at any size complete the checks: R equals the Cholesky factor of
Z^T A Z (eq. (1): Z^T A Z = R^T Q^T A Q R = R^T R), and the first row of R and
q_1 equal their definitions r_11 = ||z_1||_A, r_1j = (A z_1)^T z_j / r_11,
q_1 = z_1 / r_11, evaluated one by one.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_1703_10440_gb300 import mgsa  # noqa: E402

VARIANTS = ["naive", "ha", "hp"]


@pytest.fixture(scope="module")
def handle():
    h = mgsa.Handle(0)
    yield h
    h.close()


def to_dev(A, Z):
    d = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)
    Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to(d).T
    m = len(A[0]) - 1
    Asp = torch.sparse_csr_tensor(Ad[0].to(torch.int64), Ad[1].to(torch.int64), Ad[2], size=(m, m))
    return Ad, Zd, Asp


def metrics(Asp, Zd, Q, R):
    Q = Q if torch.is_tensor(Q) else torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    R = R if torch.is_tensor(R) else torch.from_numpy(np.ascontiguousarray(R)).cuda()
    rep = (torch.linalg.norm(Zd - Q @ R) / torch.linalg.norm(Zd)).item()
    AQ = torch.sparse.mm(Asp, Q.contiguous())
    G = Q.T @ AQ
    loss = torch.linalg.norm(G - torch.eye(G.shape[0], dtype=G.dtype, device=G.device)).item()
    return rep, loss


def chol_gram(Asp, Zd):
    AZ = torch.sparse.mm(Asp, Zd.contiguous())
    G = Zd.T @ AZ
    G = 0.5 * (G + G.T)
    return torch.linalg.cholesky(G).T  # upper factor


def first_row(A, Z):
    rowptr, col, val = A
    z1 = Z[:, 0]
    x1 = oracle.csr_mv(A, z1)
    r11 = np.sqrt(np.dot(z1, x1))
    return r11, (x1 @ Z) / r11


def against_oracle(A, Z, v, Q, R, well_conditioned):
    """Element-wise parity of the CUDA result (Q on the device, R) with the
    same form of the oracle; returns the oracle's (Q, R)."""
    Qo, Ro, info, _ = oracle.mgs_par(A, Z, v)
    assert info == 0
    Rg = R.cpu().numpy()
    kR = np.linalg.cond(Ro)
    rel = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
    if well_conditioned:
        assert rel <= 1e-10, (v, rel)
    assert np.abs(Rg - Ro).max() <= 1e-9 * kR * np.abs(Ro).max(), v
    Qg = Q.cpu().numpy()
    dq = np.abs(Qg - Qo).max()
    assert dq <= 1e-9 * kR * np.abs(Qo).max(), (v, dq)
    print(f"{v}: |R-Ro|_F/|R|_F = {rel:.2e}, max|Q-Qo| = {dq:.2e}, kappa(R) = {kR:.2e}")
    del Qg
    return Qo, Ro


def test_poisson2d_full_all_variants(handle):
    A, Z = W.poisson2d()  # m = 262144, n = 64, kappa(Z) ~ 1e6
    Ad, Zd, Asp = to_dev(A, Z)
    r11, r1 = first_row(A, Z)
    for v in VARIANTS:
        Q, R = handle.qr(Ad, Zd, v)
        assert handle.info() == (mgsa.MGSA_OK, 0)
        rep_g, loss_g = metrics(Asp, Zd, Q, R)
        Qo, Ro = against_oracle(A, Z, v, Q, R, well_conditioned=False)
        rep_o, loss_o = metrics(Asp, Zd, Qo, Ro)
        print(f"poisson2d {v}: repr {rep_g:.3e} (oracle {rep_o:.3e}), loss {loss_g:.3e} (oracle {loss_o:.3e})")
        assert rep_g <= max(1e-13, 10 * rep_o), (v, rep_g, rep_o)
        assert loss_g <= max(1e-12, 10 * loss_o), (v, loss_g, loss_o)
        Rg = R.cpu().numpy()
        assert np.all(np.tril(Rg, -1) == 0.0) and np.all(np.diag(Rg) > 0)
        assert abs(Rg[0, 0] - r11) <= 1e-13 * r11
        assert np.abs(Rg[0, :] - r1).max() <= 1e-12 * np.abs(r1).max()
        del Q, R, Qo


def test_varcoef3d_full(handle):
    A, Z = W.varcoef3d()  # m = 2097152, n = 128, kappa(Z) ~ 1
    Ad, Zd, Asp = to_dev(A, Z)
    Rc = chol_gram(Asp, Zd)
    r11, r1 = first_row(A, Z)
    for v in VARIANTS:
        Q, R = handle.qr(Ad, Zd, v)
        assert handle.info() == (mgsa.MGSA_OK, 0)
        rep_g, loss_g = metrics(Asp, Zd, Q, R)
        assert (torch.linalg.norm(R - Rc) / torch.linalg.norm(Rc)).item() <= 1e-8, v
        Rg = R.cpu().numpy()
        assert np.all(np.tril(Rg, -1) == 0.0) and np.all(np.diag(Rg) > 0)
        assert abs(Rg[0, 0] - r11) <= 1e-13 * r11
        assert np.abs(Rg[0, :] - r1).max() <= 1e-12 * np.abs(r1).max()
        q1 = Q[:, 0].cpu().numpy()
        assert np.abs(q1 - Z[:, 0] / r11).max() <= 1e-14 * np.abs(Z[:, 0]).max() / r11
        Qo, Ro = against_oracle(A, Z, v, Q, R, well_conditioned=True)
        del Q, R
        rep_o, loss_o = metrics(Asp, Zd, Qo, Ro)
        del Qo
        print(f"varcoef3d {v}: repr {rep_g:.3e} (oracle {rep_o:.3e}), loss {loss_g:.3e} (oracle {loss_o:.3e})")
        assert rep_g <= max(1e-13, 10 * rep_o), (v, rep_g, rep_o)
        assert loss_g <= max(1e-12, 10 * loss_o), (v, loss_g, loss_o)
