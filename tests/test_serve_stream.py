"""Host-side properties of the served request stream (no GPU)."""
import numpy as np

from paper_1703_10440_gb300.serve import poisson_arrivals


def test_sizes_do_not_depend_on_rate():
    lo = poisson_arrivals(50.0, 2.0)
    hi = poisson_arrivals(400.0, 2.0)
    k = min(len(lo), len(hi))
    assert k > 50
    assert [(r.m, r.n, r.kind) for r in lo[:k]] == [(r.m, r.n, r.kind) for r in hi[:k]]


def test_stream_statistics():
    reqs = poisson_arrivals(2000.0, 5.0)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < 5.0
    assert abs(len(reqs) / 5.0 - 2000.0) < 5 * np.sqrt(2000.0 / 5.0) * 5  # Poisson count
    m = np.array([r.m for r in reqs])
    n = np.array([r.n for r in reqs])
    assert m.min() >= 1000 and m.max() <= 1_000_000
    assert abs(np.mean(np.log(m)) - 0.5 * (np.log(1e3) + np.log(1e6))) < 0.1  # log-uniform
    assert n.min() >= 8 and n.max() <= 128
    kinds = [r.kind for r in reqs]
    assert 0.45 < kinds.count("laplace") / len(kinds) < 0.55


class _GangStub:
    """The fields of Server that the gang policy reads (no GPU)."""

    large_ctas = 136
    rows_per_cta = 4096
    sms = 152
    variant = "hp"
    slice_ms = 2.0

    def __init__(self, fill="prefix"):
        self.gang_fill = fill

    def _step_s(self, r, i, ctas=0):
        from paper_1703_10440_gb300.serve import Server

        return Server._step_s(self, r, i, ctas)


def _req(m, n=64):
    from paper_1703_10440_gb300.serve import Request

    return Request(0, m, n, "banded", 0.0)


def _gangs(cands, fill="prefix"):
    from paper_1703_10440_gb300.serve import Server

    return Server._gangs(_GangStub(fill), cands)


def test_gangs_fit_the_large_part_and_respect_slab_bounds():
    for cands in ([_req(1_000_000)], [_req(3000)], [_req(10_000), _req(1_000_000)],
                  [_req(m) for m in (20_000, 40_000, 80_000, 500_000, 900_000)], [_req(2000) for _ in range(80)]):
        for fill in ("prefix", "greedy"):
            g = _gangs(cands, fill)
            assert 1 <= len(g) <= 64
            assert sum(c for _, c in g) <= 136
            for r, c in g:
                assert 1 <= c <= max(1, -(-r.m // 128))  # at least 128 rows per CTA
            assert [r for r, _ in g] == [r for r in cands if any(r is x for x, _ in g)]  # order kept


def test_gangs_latency_and_throughput_sizing():
    # Alone, a request takes every CTA it can use.
    (r, c), = _gangs([_req(1_000_000)])
    assert c == 136
    (r, c), = _gangs([_req(3000)])
    assert c == 24  # ceil(3000 / 128): the smallest slab
    # Without a backlog the request closest to done wants one CTA per 1024
    # rows.  "prefix" then stops at the big request, which does not fit the
    # rest, and the small one gets every CTA it can use; "greedy" gives the big
    # one the rest, since one of its steps fits a slice on 126 CTAs.
    g = _gangs([_req(10_000), _req(1_000_000)], "prefix")
    assert [c for _, c in g] == [79]
    g = _gangs([_req(10_000), _req(1_000_000)], "greedy")
    assert [c for _, c in g] == [10, 126]
    # With a backlog, one CTA per 4096 rows; "prefix" stops at the first
    # request that does not fit, "greedy" squeezes one whose step fits a slice.
    cands = [_req(m) for m in (30_000, 50_000, 200_000, 1_000_000)]
    g = _gangs(cands, "prefix")
    assert [r.m for r, _ in g] == [30_000, 50_000, 200_000] and sum(c for _, c in g) == 136
    g = _gangs(cands, "greedy")
    assert [r.m for r, _ in g] == [30_000, 50_000, 200_000, 1_000_000] and sum(c for _, c in g) == 136
