"""Serving: a request loop with continuous batching over the C ABI.

Requests (n, k, alpha, seed) arrive over time.  A request is admitted when its
device-memory estimate (workspace + pairs for the expected edge count n k / 2
with slack) fits in what the budget has left; admitted work runs on one of
several workers, each a host thread with its own CUDA stream, so that the
generations of different requests overlap on the device (the library calls
release the interpreter lock while they wait for their stream).  A worker that
takes a small request also takes the small requests queued directly behind it,
as long as they fit, and generates them together with one rhg_generate_batch
call.  Admission is first come, first served: a request that does not fit
waits for memory, and the requests behind it wait too.

The scheduling is independent of the GPU: the executor (estimate, single,
batch) can be replaced, which the host tests do.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass


@dataclass
class Request:
    rid: int
    n: int
    k: float
    alpha: float
    seed: int
    arrival: float = 0.0  # seconds on the server's clock (time.perf_counter)


@dataclass
class Completion:
    rid: int
    m: int
    R: float
    arrival: float
    start: float
    end: float
    batch_size: int          # 1: alone; >1: generated in a batch of that many requests
    pairs: object = None     # the (m, 2) pairs when the server keeps results

    @property
    def latency(self) -> float:
        return self.end - self.arrival


class GpuExecutor:
    """Runs requests with the library: one graph with rhg_generate_pairs, a group
    of small graphs with rhg_generate_batch."""

    def __init__(self, keep_results: bool = False):
        from . import (batch_params, batch_workspace_bytes, estimate_capacity, generate_batch, generate_pairs,
                       make_params, workspace_bytes)
        self._bp, self._bwb, self._est = batch_params, batch_workspace_bytes, estimate_capacity
        self._gb, self._gp, self._mp, self._wb = generate_batch, generate_pairs, make_params, workspace_bytes
        self.keep = keep_results

    def estimate(self, r: Request) -> int:
        return int(self._wb(self._mp(r.n, r.k, r.alpha, r.seed), 0)) + 8 * self._est(r.n, r.k)

    def estimate_batch(self, rs) -> int:
        return int(self._bwb(self._bp([(r.n, r.k, r.alpha, r.seed) for r in rs]))) + \
            8 * sum(self._est(r.n, r.k) for r in rs)

    def single(self, r: Request, stream):
        pairs, res = self._gp(r.n, r.k, r.alpha, r.seed, stream=stream)
        return [(int(res.m), float(res.R), pairs if self.keep else None)]

    def batch(self, rs, stream):
        views, results, _ = self._gb([(r.n, r.k, r.alpha, r.seed) for r in rs], stream=stream)
        return [(int(res.m), float(res.R), v if self.keep else None) for v, res in zip(views, results)]


@dataclass
class _Work:
    reqs: list
    reserve: int


class Server:
    """budget_bytes: device memory the admitted requests may hold at once;
    workers: concurrent generations; small_n / batch_points: requests with
    n <= small_n are grouped, up to batch_points points per group."""

    def __init__(self, executor=None, budget_bytes: int = 120 * 10**9, workers: int = 4, small_n: int = 100_000,
                 batch_points: int = 4_000_000, batch_max: int = 256, use_cuda_streams: bool = True):
        self.ex = executor if executor is not None else GpuExecutor()
        self.budget = int(budget_bytes)
        self.free = int(budget_bytes)
        self.small_n, self.batch_points, self.batch_max = small_n, batch_points, batch_max
        self.queue = deque()
        self.cv = threading.Condition()
        self.done: list[Completion] = []
        self.errors: list[BaseException] = []
        self.closing = False
        self.peak_reserved = 0
        self.admitted: list[list[int]] = []  # request ids of each admitted piece of work, in order
        self.use_cuda_streams = use_cuda_streams
        self.threads = [threading.Thread(target=self._worker, daemon=True) for _ in range(workers)]
        for t in self.threads:
            t.start()

    # ---------------------------------------------------------------- clients
    def submit(self, r: Request):
        need = self.ex.estimate(r)
        if need > self.budget:
            raise ValueError(f"request {r.rid} needs {need} bytes, more than the budget {self.budget}")
        with self.cv:
            self.queue.append(r)
            self.cv.notify_all()

    def close(self, timeout: float | None = None):
        """Waits until every submitted request has completed, then stops the workers."""
        with self.cv:
            self.closing = True
            self.cv.notify_all()
        for t in self.threads:
            t.join(timeout)
        if self.errors:
            raise self.errors[0]

    # ------------------------------------------------------------- scheduling
    def _take(self):
        """Admits the head of the queue (and small followers) if it fits; else None."""
        head = self.queue[0]
        need = self.ex.estimate(head)
        if need > self.free:
            return None
        reqs = [head]
        if head.n <= self.small_n:
            pts = head.n
            i = 1
            while i < len(self.queue) and len(reqs) < self.batch_max:
                r = self.queue[i]
                if r.n > self.small_n or pts + r.n > self.batch_points:
                    break
                reqs.append(r)
                pts += r.n
                i += 1
            if len(reqs) > 1:
                need = self.ex.estimate_batch(reqs)
                while need > self.free and len(reqs) > 1:
                    reqs.pop()
                    need = self.ex.estimate_batch(reqs) if len(reqs) > 1 else self.ex.estimate(head)
                if need > self.free:
                    return None
        for _ in reqs:
            self.queue.popleft()
        self.free -= need
        self.peak_reserved = max(self.peak_reserved, self.budget - self.free)
        self.admitted.append([r.rid for r in reqs])
        return _Work(reqs, need)

    def _worker(self):
        stream = None
        if self.use_cuda_streams:
            import torch
            stream = torch.cuda.Stream()
        while True:
            with self.cv:
                work = None
                while work is None:
                    if self.queue:
                        work = self._take()
                        if work is not None:
                            break
                    elif self.closing:
                        return
                    self.cv.wait()
            start = time.perf_counter()
            try:
                if stream is not None:
                    import torch
                    with torch.cuda.stream(stream):
                        out = self._run(work, stream)
                else:
                    out = self._run(work, stream)
            except BaseException as e:  # reported by close()
                with self.cv:
                    self.errors.append(e)
                    self.free += work.reserve
                    self.cv.notify_all()
                continue
            end = time.perf_counter()
            with self.cv:
                for r, (m, R, pairs) in zip(work.reqs, out):
                    self.done.append(Completion(r.rid, m, R, r.arrival, start, end, len(work.reqs), pairs))
                self.free += work.reserve
                self.cv.notify_all()

    def _run(self, work: _Work, stream):
        if len(work.reqs) == 1:
            return self.ex.single(work.reqs[0], stream)
        return self.ex.batch(work.reqs, stream)


def percentile(xs, q: float) -> float:
    """The q-quantile (0..1) by linear interpolation between order statistics."""
    s = sorted(xs)
    if not s:
        return float("nan")
    pos = q * (len(s) - 1)
    i = int(pos)
    f = pos - i
    return s[i] if i + 1 >= len(s) else s[i] * (1 - f) + s[i + 1] * f


def replay(server: Server, requests, clock=time.perf_counter, sleep=time.sleep):
    """Submits the requests at their arrival offsets (seconds from now), waits
    for all, and returns the completions sorted by request id."""
    t0 = clock()
    for r in sorted(requests, key=lambda r: r.arrival):
        wait = t0 + r.arrival - clock()
        if wait > 0:
            sleep(wait)
        r.arrival = t0 + r.arrival
        server.submit(r)
    server.close()
    return sorted(server.done, key=lambda c: c.rid)


def poisson_requests(count: int, rate: float, seed: int = 5, first_rid: int = 0):
    """The served workload: n = floor(10^U(4, 7)), k uniform in 8..64, alpha
    uniform in [0.6, 1.2], seed 10^6 + request number, arrivals of a Poisson
    process of the given rate (per second), drawn by numpy's PCG64."""
    import numpy as np
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for j in range(count):
        out.append(Request(first_rid + j, int(10 ** rng.uniform(4, 7)), int(rng.integers(8, 65)),
                           float(rng.uniform(0.6, 1.2)), 10**6 + first_rid + j, float(t[j])))
    return out
