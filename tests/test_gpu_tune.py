"""The launch parameters the autotuner searches, on the GPU: the panel width of
the block product changes nothing (every column's sums are the same), the row
mode changes only rounding (parity with the oracle holds either way), and the
tuner's chosen setting is one of the timed candidates, is applied to the
handle, survives a round trip through its cache, and gives results within
the parity gates."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa, tune  # noqa: E402
from paper_1703_10440_gb300.batch import Batch  # noqa: E402


@pytest.fixture(scope="module")
def handle():
    h = mgsa.Handle(0)
    yield h
    h.close()


def dev(A, Z):
    d = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in A)
    return Ad, torch.from_numpy(np.ascontiguousarray(np.asarray(Z).T)).to(d).T


def run(h, A, Z, variant, **params):
    tune.apply(h.h, params)
    try:
        Ad, Zd = dev(A, Z)
        Q, R = h.qr(Ad, Zd, variant)
        assert h.info() == (mgsa.MGSA_OK, 0)
        return Q.cpu().numpy(), R.cpu().numpy()
    finally:
        tune.reset(h.h, params)


def check(A, Z, variant, Q, R):
    Qo, Ro, info, _, _ = oracle.mgs(A, Z, variant, "row")
    assert info == 0
    assert oracle.repr_error(Z, Q, R) <= max(1e-13, 10 * oracle.repr_error(Z, Qo, Ro))
    assert oracle.orth_loss(A, Q) <= max(1e-12, 10 * oracle.orth_loss(A, Qo))
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10


@pytest.mark.parametrize("case", ["banded", "denseband"])
def test_panel_width_changes_nothing(handle, case):
    A, Z = W.banded(20011, 21, seed=5) if case == "banded" else W.denseband(2000, 24, hb=100)
    Q4, R4 = run(handle, A, Z, "hp", spmm_panel=4)
    Q8, R8 = run(handle, A, Z, "hp", spmm_panel=8)
    assert np.array_equal(Q4, Q8) and np.array_equal(R4, R8)


@pytest.mark.parametrize("variant", ["naive", "ha", "hp"])
@pytest.mark.parametrize("row_mode", [1, 2])
def test_row_mode_parity(handle, variant, row_mode):
    for A, Z in (W.banded(5003, 12, seed=6), W.denseband(2000, 24, hb=100)):
        Q, R = run(handle, A, Z, variant, row_mode=row_mode)
        check(A, Z, variant, Q, R)


@pytest.mark.parametrize("variant", ["ha", "hp"])
def test_tune_qr(handle, variant, tmp_path):
    A, Z = W.banded(60000, 16, seed=15)
    Ad, Zd = dev(A, Z)
    t = tune.Tuner(str(tmp_path / "tune.json"))
    rec = t.tune_qr(handle, Ad, Zd, variant, reps=2)
    try:
        space = tune.candidates(tune.SINGLE_SPACE, variant, None)
        assert [tr["params"] for tr in rec["trials"]] == space
        assert rec["ms"] == min(tr["ms"] for tr in rec["trials"]) > 0
        Q, R = handle.qr(Ad, Zd, variant)  # runs with the chosen setting applied
        assert handle.info() == (mgsa.MGSA_OK, 0)
        check(A, Z, variant, Q.cpu().numpy(), R.cpu().numpy())
    finally:
        tune.reset(handle.h, list(tune.SINGLE_SPACE))
    t.save()
    key = tune.bucket_key(torch.cuda.get_device_name(), variant, 60000, 16, len(A[1]))
    assert tune.Tuner(str(tmp_path / "tune.json")).lookup(key) == rec["params"]


def test_tune_batched(handle, tmp_path):
    inst = [W.banded(m, n, seed=100 + k) for k, (m, n) in enumerate([(3000, 40), (1200, 16), (700, 8), (5000, 24)])]
    b = Batch(inst, ["hp", "ha", "hp", "naive"])
    t = tune.Tuner(str(tmp_path / "tune.json"))
    rec = t.tune_batched(handle, b, reps=2)
    try:
        assert rec["params"] in tune.candidates(tune.BATCH_SPACE, "hp")
        b.run(handle.h)
        infos = b.infos()
        assert np.all(infos == 0)
        for k, ((A, Z), v) in enumerate(zip(inst, ["hp", "ha", "hp", "naive"])):
            Q, R, _ = b.result(k)
            check(A, Z, v, Q, R)
    finally:
        tune.reset(handle.h, list(tune.BATCH_SPACE))
