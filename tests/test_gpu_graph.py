"""mgsa_qr (one cooperative launch) inside a CUDA graph: after mgsa_reserve the
call allocates nothing, so it can be captured; replays with new contents of
the captured Z buffer give bitwise the results of direct calls, and the
status copied by mgsa_copy_info inside the graph is that of each replay."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402

FORMS = ["naive", "ha", "hp", "cgs_ha", "cgs_hp"]


@pytest.mark.parametrize("variant", FORMS)
def test_qr_graph_capture_and_replay(variant):
    d = torch.device("cuda")
    A, Z0 = W.banded(30011, 12, seed=31)
    m, n = Z0.shape
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)
    h = mgsa.Handle(0)
    try:
        v = mgsa.VARIANTS[variant]
        mgsa.mgsa_reserve(h.h, m, n, v)
        Zbuf = torch.empty((n, m), dtype=torch.float64, device=d).T
        Q = torch.empty((n, m), dtype=torch.float64, device=d).T
        R = torch.empty((n, n), dtype=torch.float64, device=d).T
        info = torch.zeros(2, dtype=torch.int32, device=d)
        csr = mgsa.make_csr(m, Ad[1].numel(), *Ad)
        s = torch.cuda.Stream(d)
        Zbuf.copy_(torch.from_numpy(np.ascontiguousarray(Z0.T)).to(d).T)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            st = mgsa.mgsa_qr(h.h, csr, Zbuf, m, n, m, v, Q, m, R, n, s)
            mgsa.mgsa_copy_info(h.h, info, s)
        assert st == mgsa.MGSA_OK, mgsa.mgsa_last_error()
        rng = np.random.Generator(np.random.PCG64(5))
        for k in range(3):
            Zk = Z0 if k == 0 else rng.standard_normal((m, n))
            if k == 2:
                Zk = Zk.copy()
                Zk[:, 5] = 0.0  # breakdown at column 6
            Zbuf.copy_(torch.from_numpy(np.ascontiguousarray(Zk.T)).to(d).T)
            g.replay()
            torch.cuda.synchronize()
            got_info = info.cpu().tolist()
            Qd, Rd = h.qr(Ad, torch.from_numpy(np.ascontiguousarray(Zk.T)).to(d).T, variant)
            st_d, info_d = h.info()
            if k < 2:
                assert got_info == [0, 0] and (st_d, info_d) == (mgsa.MGSA_OK, 0)
                assert torch.equal(Q, Qd) and torch.equal(R, Rd)
            else:
                assert got_info == [mgsa.MGSA_ERR_BREAKDOWN, 6] and (st_d, info_d) == (mgsa.MGSA_ERR_BREAKDOWN, 6)
    finally:
        h.close()
