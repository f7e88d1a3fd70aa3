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
