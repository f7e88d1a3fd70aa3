"""The continuous-batching server: every request's result is the same when it
is served alone and when it is served in a mix of concurrent requests of
different sizes (batched and whole-GPU launches interleaved), and agrees with
the CPU oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402
from paper_1703_10440_gb300.serve import KeepingServer, Request, poisson_arrivals  # noqa: E402


@pytest.fixture(scope="module")
def handle():
    h = mgsa.Handle(0)
    yield h
    h.close()


def make_requests():
    reqs = poisson_arrivals(rate=400.0, duration=0.1, m_lo=1e3, m_hi=6e4, n_lo=8, n_hi=48)
    assert len(reqs) >= 20
    return reqs


def fresh(reqs):
    return [Request(r.rid, r.m, r.n, r.kind, r.arrival, r.seed) for r in reqs]


def test_served_alone_equals_in_mix(handle):
    reqs = make_requests()
    # small_work splits the mix between the batched kernel and whole-GPU launches
    mix = KeepingServer(handle.h, "hp", budget_bytes=8e9, small_work=5e6, max_m=60000, max_n=48)
    stats = mix.run(fresh(reqs), realtime=True)
    assert stats["ok"] == len(reqs)
    assert 0 < stats["small"] < len(reqs)
    alone = KeepingServer(handle.h, "hp", budget_bytes=8e9, small_work=5e6, max_m=60000, max_n=48)
    for r in fresh(reqs):
        alone.run([Request(r.rid, r.m, r.n, r.kind, 0.0, r.seed)], realtime=False)
    for rid, (Q, R, info) in mix.results.items():
        Qa, Ra, info_a = alone.results[rid]
        assert info == info_a == 0
        assert np.linalg.norm(R - Ra) / np.linalg.norm(Ra) <= 1e-12
        assert np.abs(Q - Qa).max() <= 1e-10 * np.abs(Qa).max()


def test_served_results_match_oracle(handle):
    from workloads import device as wd

    reqs = fresh(make_requests())[:6]
    srv = KeepingServer(handle.h, "ha", budget_bytes=8e9, small_work=5e6, max_m=60000, max_n=48)
    srv.run(reqs, realtime=False)
    for r in reqs:
        A, Z, m = wd.request_inputs(r.kind, r.m, r.n, r.seed, r.rid, torch.device("cuda"))
        A = tuple(t.cpu().numpy() for t in A)
        Z = np.asfortranarray(Z.cpu().numpy())
        Q, R, info = srv.results[r.rid]
        Qo, Ro, oinfo, _, _ = oracle.mgs(A, Z, "ha", "row")
        assert info == 0 and oinfo == 0
        assert oracle.repr_error(Z, Q, R) <= max(1e-13, 10 * oracle.repr_error(Z, Qo, Ro))
        assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10


def test_admission_under_a_tight_budget(handle):
    reqs = fresh(make_requests())[:10]
    srv = KeepingServer(handle.h, "hp", budget_bytes=2.5e8, small_work=5e6, max_m=60000, max_n=48)
    stats = srv.run(reqs, realtime=False)
    assert stats["ok"] == len(reqs)
    biggest = max(srv._bytes(r) for r in reqs)
    assert stats["peak_bytes"] <= 2.5e8 + biggest


def test_partitioned_sms(handle):
    """small_ctas: large requests on the other SMs, small ones on their own
    stream and handle at the same time.  Each result is the same alone and in
    the mix (same partition); small requests are bitwise the results of an
    unpartitioned server (one CTA runs one instance either way), large ones
    agree with it to rounding; and all match the oracle's invariants."""
    reqs = make_requests()
    kw = dict(budget_bytes=8e9, small_work=5e6, max_m=60000, max_n=48)
    mix = KeepingServer(handle.h, "hp", small_ctas=16, **kw)
    try:
        stats = mix.run(fresh(reqs), realtime=True)
        assert stats["ok"] == len(reqs) and 0 < stats["small"] < len(reqs)
        alone = KeepingServer(handle.h, "hp", small_ctas=16, **kw)
        try:
            for r in fresh(reqs):
                alone.run([Request(r.rid, r.m, r.n, r.kind, 0.0, r.seed)], realtime=False)
        finally:
            alone.close()
    finally:
        mix.close()
    plain = KeepingServer(handle.h, "hp", **kw)
    plain.run(fresh(reqs), realtime=False)
    for r in reqs:
        Q, R, info = mix.results[r.rid]
        Qa, Ra, _ = alone.results[r.rid]
        Qp, Rp, _ = plain.results[r.rid]
        assert info == 0
        assert np.linalg.norm(R - Ra) / np.linalg.norm(Ra) <= 1e-12
        assert np.abs(Q - Qa).max() <= 1e-10 * np.abs(Qa).max()
        if r.m * r.n ** 2 <= 5e6:
            assert np.array_equal(Q, Qp) and np.array_equal(R, Rp)
        else:
            assert np.linalg.norm(R - Rp) / np.linalg.norm(Rp) <= 1e-10
    # the caller's handle is back to its default CTA count
    A, Z = W.tridiag(3000, 4)
    d = torch.device("cuda")
    Ad = tuple(torch.from_numpy(np.ascontiguousarray(x)).to(d) for x in A)
    Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to(d).T
    handle.set_param(mgsa.MGSA_PARAM_CLUSTER, 1)  # a whole-GPU launch, where the CTA count shows
    try:
        Q1, R1 = handle.qr(Ad, Zd, "hp")
        assert handle.info() == (mgsa.MGSA_OK, 0)
    finally:
        handle.set_param(mgsa.MGSA_PARAM_CLUSTER, 0)
    h2 = mgsa.Handle(0)
    h2.set_param(mgsa.MGSA_PARAM_CLUSTER, 1)
    Q2, R2 = h2.qr(Ad, Zd, "hp")
    assert h2.info() == (mgsa.MGSA_OK, 0)
    h2.close()
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)


def test_shortest_work_first_window(handle):
    """max_large_inflight: large requests wait on the host and are launched
    least work first, at most two at a time; results are unchanged."""
    reqs = make_requests()
    kw = dict(budget_bytes=8e9, small_work=5e6, max_m=60000, max_n=48)
    srv = KeepingServer(handle.h, "hp", small_ctas=16, max_large_inflight=2, **kw)
    try:
        stats = srv.run(fresh(reqs), realtime=True)
    finally:
        srv.close()
    assert stats["ok"] == len(reqs)
    plain = KeepingServer(handle.h, "hp", small_ctas=16, **kw)
    try:
        plain.run(fresh(reqs), realtime=False)
    finally:
        plain.close()
    for r in reqs:
        Q, R, _ = srv.results[r.rid]
        Qp, Rp, _ = plain.results[r.rid]
        assert np.array_equal(Q, Qp) and np.array_equal(R, Rp)


@pytest.mark.parametrize("variant", ["ha", "hp"])
def test_time_sliced_large_requests(handle, variant):
    """slice_ms with large_mode "slices": large requests run as whole-GPU time
    slices on pool handles, least remaining work first; every result is
    bitwise that of the unsliced server with the same SM partition."""
    reqs = make_requests()
    kw = dict(budget_bytes=8e9, small_work=5e6, max_m=60000, max_n=48, small_ctas=16)
    sl = KeepingServer(handle.h, variant, slice_ms=0.05, large_handles=2, large_mode="slices", **kw)
    try:
        stats = sl.run(fresh(reqs), realtime=True)
    finally:
        sl.close()
    assert stats["ok"] == len(reqs)
    assert stats["launches"] > stats["small"] and 0 < stats["small"] < len(reqs)
    handle.set_param(mgsa.MGSA_PARAM_CLUSTER, 1)  # slices run on the whole GPU (its large part)
    plain = KeepingServer(handle.h, variant, **kw)
    try:
        plain.run(fresh(reqs), realtime=False)
    finally:
        plain.close()
        handle.set_param(mgsa.MGSA_PARAM_CLUSTER, 0)
    for r in reqs:
        Q, R, info = sl.results[r.rid]
        Qp, Rp, infop = plain.results[r.rid]
        assert info == infop == 0
        assert np.array_equal(Q, Qp) and np.array_equal(R, Rp), r.rid


@pytest.mark.parametrize("variant", ["naive", "hp"])
def test_grouped_slices_alone_equal_in_mix(handle, variant):
    """slice_ms with the default large_mode "group": large requests share
    grouped launches (a gang of CTAs each, sized by the load), up to two
    launches queued.  Each result is the same alone and in the mix within the
    tolerance of the other serving tests (gang sizes, hence reduction trees,
    differ with the load), and meets the oracle's gates."""
    from workloads import device as wd

    reqs = make_requests()
    kw = dict(budget_bytes=8e9, small_work=5e6, max_m=60000, max_n=48, small_ctas=16, slice_ms=0.2,
              max_large_inflight=2)
    mix = KeepingServer(handle.h, variant, **kw)
    try:
        stats = mix.run(fresh(reqs), realtime=True)
    finally:
        mix.close()
    assert stats["ok"] == len(reqs) and 0 < stats["small"] < len(reqs)
    alone = KeepingServer(handle.h, variant, **kw)
    try:
        for r in fresh(reqs):
            alone.run([Request(r.rid, r.m, r.n, r.kind, 0.0, r.seed)], realtime=False)
    finally:
        alone.close()
    for r in reqs:
        Q, R, info = mix.results[r.rid]
        Qa, Ra, info_a = alone.results[r.rid]
        assert info == info_a == 0
        assert np.linalg.norm(R - Ra) / np.linalg.norm(Ra) <= 1e-12
        assert np.abs(Q - Qa).max() <= 1e-10 * np.abs(Qa).max()
    large = [r for r in reqs if r.m * r.n ** 2 > 5e6][:3]
    assert large
    for r in large:
        A, Z, _ = wd.request_inputs(r.kind, r.m, r.n, r.seed, r.rid, torch.device("cuda"))
        A = tuple(t.cpu().numpy() for t in A)
        Z = np.asfortranarray(Z.cpu().numpy())
        Q, R, _ = mix.results[r.rid]
        Qo, Ro, oinfo, _, _ = oracle.mgs(A, Z, variant, "row")
        assert oinfo == 0
        assert oracle.repr_error(Z, Q, R) <= max(1e-13, 10 * oracle.repr_error(Z, Qo, Ro))
        assert oracle.orth_loss(A, Q) <= max(1e-12, 10 * oracle.orth_loss(A, Qo))
        assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10


def test_small_requests_in_their_own_form(handle):
    """small_variant: the batched small requests run in another form than the
    large ones (here HP next to HA).  Each result meets the gates of its own
    form of the oracle, and a small result equals, bit for bit, the one of a
    server whose form is that form throughout."""
    from workloads import device as wd

    reqs = fresh(make_requests())[:12]
    kw = dict(budget_bytes=8e9, small_work=5e6, max_m=60000, max_n=48)
    srv = KeepingServer(handle.h, "ha", small_variant="hp", **kw)
    stats = srv.run(reqs, realtime=False)
    assert stats["ok"] == len(reqs) and 0 < stats["small"] < len(reqs)
    same = KeepingServer(handle.h, "hp", **kw)
    same.run(fresh(reqs), realtime=False)
    for r in reqs:
        small = r.m * r.n ** 2 <= 5e6
        form = "hp" if small else "ha"
        A, Z, _ = wd.request_inputs(r.kind, r.m, r.n, r.seed, r.rid, torch.device("cuda"))
        A = tuple(t.cpu().numpy() for t in A)
        Z = np.asfortranarray(Z.cpu().numpy())
        Q, R, info = srv.results[r.rid]
        Qo, Ro, oinfo, _, _ = oracle.mgs(A, Z, form, "row")
        assert info == 0 and oinfo == 0
        assert oracle.repr_error(Z, Q, R) <= max(1e-13, 10 * oracle.repr_error(Z, Qo, Ro))
        assert oracle.orth_loss(A, Q) <= max(1e-12, 10 * oracle.orth_loss(A, Qo))
        assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10
        if small:
            Qs, Rs, _ = same.results[r.rid]
            assert np.array_equal(Q, Qs) and np.array_equal(R, Rs), r.rid
