"""Serving loop on the host with a fake executor (no GPU): first-come admission
under the memory budget, grouping of small requests, overlap of work, and the
latency statistics."""
import threading
import time

import pytest

from paper_1606_09481_gb300.serve import Request, Server, percentile, poisson_requests, replay


class FakeExecutor:
    """estimate = n bytes; work takes n microseconds; m = 3 n."""

    def __init__(self):
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.calls = []

    def estimate(self, r):
        return r.n

    def estimate_batch(self, rs):
        return sum(r.n for r in rs) + 10

    def _work(self, rs):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.calls.append([r.rid for r in rs])
        time.sleep(sum(r.n for r in rs) * 1e-6)
        with self.lock:
            self.active -= 1
        return [(3 * r.n, 1.0, None) for r in rs]

    def single(self, r, stream):
        return self._work([r])

    def batch(self, rs, stream):
        return self._work(rs)


def test_fifo_admission_respects_budget():
    ex = FakeExecutor()
    srv = Server(ex, budget_bytes=10_000, workers=4, small_n=0, use_cuda_streams=False)
    reqs = [Request(i, 6000 if i % 3 == 0 else 2500, 8, 1.0, i, 0.0) for i in range(30)]
    for r in reqs:
        srv.submit(r)
    srv.close()
    assert [a for a in srv.admitted] == [[i] for i in range(30)]  # first come, first served
    assert srv.peak_reserved <= 10_000
    assert srv.free == 10_000
    assert sorted(c.rid for c in srv.done) == list(range(30))
    assert all(c.m == 3 * reqs[c.rid].n for c in srv.done)
    assert ex.max_active >= 2  # work overlapped


def test_small_requests_are_grouped():
    ex = FakeExecutor()
    srv = Server(ex, budget_bytes=10**9, workers=1, small_n=1000, batch_points=5000, batch_max=8,
                 use_cuda_streams=False)
    srv.submit(Request(0, 50_000, 8, 1.0, 0, 0.0))  # occupies the one worker for 50 ms
    time.sleep(0.005)
    for i in range(1, 21):
        srv.submit(Request(i, 900, 8, 1.0, i, 0.0))
    srv.close()
    groups = srv.admitted[1:]
    assert sum(len(g) for g in groups) == 20 and max(len(g) for g in groups) > 1
    assert all(len(g) <= 8 and 900 * len(g) <= 5000 for g in groups)
    assert [rid for g in groups for rid in g] == list(range(1, 21))  # order kept
    sizes = {c.rid: c.batch_size for c in srv.done}
    assert sizes[0] == 1 and max(sizes.values()) > 1


def test_request_over_budget_is_refused():
    srv = Server(FakeExecutor(), budget_bytes=100, workers=1, use_cuda_streams=False)
    with pytest.raises(ValueError):
        srv.submit(Request(0, 1000, 8, 1.0, 0, 0.0))
    srv.close()


def test_replay_and_percentiles():
    reqs = poisson_requests(40, rate=2000.0, seed=7)
    assert all(10**4 <= r.n < 10**7 and 8 <= r.k <= 64 and 0.6 <= r.alpha <= 1.2 for r in reqs)
    assert [r.seed for r in reqs] == [10**6 + j for j in range(40)]
    for r in reqs:
        r.n = r.n // 1000  # keep the fake work short
    srv = Server(FakeExecutor(), budget_bytes=10**9, workers=3, use_cuda_streams=False)
    done = replay(srv, reqs)
    assert [c.rid for c in done] == list(range(40))
    assert all(c.end >= c.start >= c.arrival - 1e-6 for c in done)
    lat = [c.latency for c in done]
    assert percentile(lat, 0.5) <= percentile(lat, 0.99) <= max(lat)
    assert percentile([1.0, 2.0, 3.0, 4.0], 0.5) == 2.5 and percentile([5.0], 0.99) == 5.0


class UnderEstimatingExecutor(FakeExecutor):
    """Requests with odd rid hold 3 n bytes of edges, but the first estimate
    (before the exact count is known) is n bytes: the first attempt runs out of
    room and gives the request back with its exact size.  Tracks the bytes the
    running work actually holds."""

    def __init__(self):
        super().__init__()
        self.held = 0
        self.max_held = 0

    def need(self, r):
        return 3 * r.n if r.rid % 2 else r.n

    def estimate(self, r):
        return max(r.n, r.m_hint)

    def estimate_batch(self, rs):
        return sum(self.estimate(r) for r in rs)

    def _work(self, rs):
        from paper_1606_09481_gb300.serve import Retry
        hold = sum(self.estimate(r) for r in rs)  # what the work allocates: its estimate, never more
        with self.lock:
            self.held += hold
            self.max_held = max(self.max_held, self.held)
            self.calls.append([r.rid for r in rs])
        time.sleep(sum(r.n for r in rs) * 1e-6)
        with self.lock:
            self.held -= hold
        return [Retry(self.need(r)) if self.need(r) > self.estimate(r) else (self.need(r), 1.0, None) for r in rs]


def test_budget_bounds_memory_when_estimates_are_short():
    ex = UnderEstimatingExecutor()
    budget = 12_000
    srv = Server(ex, budget_bytes=budget, workers=4, small_n=0, use_cuda_streams=False)
    reqs = [Request(i, 3000, 8, 1.0, i, 0.0) for i in range(24)]
    for r in reqs:
        srv.submit(r)
    srv.close()
    assert ex.max_held <= budget and srv.peak_reserved <= budget
    assert srv.retries == 12  # every odd request once
    done = {c.rid: c.m for c in srv.done}
    assert sorted(done) == list(range(24))
    assert all(done[i] == (9000 if i % 2 else 3000) for i in range(24))
    assert srv.free == budget


def test_retry_larger_than_the_budget_is_an_error():
    ex = UnderEstimatingExecutor()
    srv = Server(ex, budget_bytes=5000, workers=1, small_n=0, use_cuda_streams=False)
    srv.submit(Request(1, 3000, 8, 1.0, 1, 0.0))  # exact size 9000 > budget
    with pytest.raises(ValueError):
        srv.close()


def test_grouping_looks_past_a_large_request():
    ex = FakeExecutor()
    srv = Server(ex, budget_bytes=10**9, workers=1, small_n=1000, batch_points=5000, batch_max=8,
                 use_cuda_streams=False)
    srv.submit(Request(0, 50_000, 8, 1.0, 0, 0.0))  # occupies the one worker for 50 ms
    time.sleep(0.005)
    srv.submit(Request(1, 900, 8, 1.0, 1, 0.0))
    srv.submit(Request(2, 20_000, 8, 1.0, 2, 0.0))  # large, between small ones
    for i in range(3, 7):
        srv.submit(Request(i, 900, 8, 1.0, i, 0.0))
    srv.close()
    assert srv.admitted[1] == [1, 3, 4, 5, 6]  # the small ones grouped across the large one
    assert srv.admitted[2] == [2]
