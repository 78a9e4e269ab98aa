"""Host logic of the serving loop (no GPU): topology cache, admission, request stream."""
import numpy as np

from paper_2503_13075_gb300 import serving as sv


class FakeTopo:
    def __init__(self, n):
        self.n = n
        self.closed = False

    def close(self):
        self.closed = True


def test_cache_lru_eviction_and_budget():
    made = []

    def make(n, i, j):
        t = FakeTopo(n)
        made.append(t)
        return t

    c = sv.TopologyCache(100, make, lambda t: t.n)
    a = c.get("a", (40, None, None))
    b = c.get("b", (40, None, None))
    assert c.get("a", (40, None, None)) is a and c.hits == 1
    d = c.get("d", (40, None, None))  # evicts the least recently used ("b")
    assert b.closed and not a.closed and c.evictions == 1
    assert set(c.entries) == {"a", "d"} and c.used == 80
    # a topology that cannot fit even alone is rejected, nothing evicted
    assert c.get("huge", (150, None, None)) is None and set(c.entries) == {"a", "d"}
    # reserve for the request's buffers counts against the budget
    assert c.get("r", (30, None, None), reserve=80) is None


def test_request_stream_shape():
    reqs, pool = sv.make_requests(400, rate_hz=2000.0, seed=7, n_topologies=6, lo=20, hi=2000)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) >= 0)
    rate = len(t) / t[-1]
    assert 1500 < rate < 2600  # Poisson at 2000 / s
    sizes = sorted({r.n_atoms for r in reqs})
    assert all(20 <= n <= 2000 for n in sizes) and len(sizes) <= 6
    assert len({r.key for r in reqs}) == len(sizes)
    # coordinates are fresh per request, topology shared
    same = [r for r in reqs if r.key == reqs[0].key]
    if len(same) > 1:
        assert not np.array_equal(same[0].x_unc, same[1].x_unc)
        assert np.array_equal(same[0].atom_i, same[1].atom_i)


def test_violation_report():
    x = np.array([[0.0, 0, 0], [0.1, 0, 0]])
    assert sv.max_relative_violation(x, np.array([0]), np.array([1]), np.array([0.1])) < 1e-15
    assert abs(sv.max_relative_violation(x, np.array([0]), np.array([1]), np.array([0.2])) - 0.75) < 1e-12
