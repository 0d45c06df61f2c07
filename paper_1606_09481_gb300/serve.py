"""Serving: a request loop with continuous batching over the C ABI.

Requests (n, k, alpha, seed) arrive over time.  A request is admitted when its
device-memory estimate (workspace + pairs for the expected edge count n k / 2
with slack) fits in what the budget has left; admitted work runs on one of
several workers, each a host thread with its own CUDA stream, so that the
generations of different requests overlap on the device (the library calls
release the interpreter lock while they wait for their stream).  A worker that
takes a small request also takes the small requests queued directly behind it,
as long as they fit, and generates them together with one rhg_generate_batch
call; it looks for them among the first `lookahead` queued requests, so a large
request in between does not stop the grouping (the large one is still admitted
in its turn).  Admission is first come, first served: a request that does not
fit waits for memory, and the requests behind it wait too.

The budget is a bound on what admitted work holds: the executor never
allocates more than the estimate it was admitted with.  When a graph has more
edges than its estimate has room for, the executor gives the request back with
its exact edge count (Retry); the server releases the reservation and puts the
request back at the head of the queue with that count, so that its next
admission reserves exactly what it needs.

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
    m_hint: int = 0       # exact edge count, known after an attempt that ran out of room
    attempts: int = 0


@dataclass
class Retry:
    """An executor's answer for a request whose graph had more edges (m) than the
    room its estimate reserved."""
    m: int


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
    of small graphs with rhg_generate_batch.  Device memory never exceeds the
    estimate: the workspace and a pair buffer of capacity() pairs."""

    def __init__(self, keep_results: bool = False):
        from . import (OVERFLOW, RhgError, allocate_batch, allocate_pairs, batch_params, batch_workspace_bytes,
                       estimate_capacity, generate_pairs, make_params, run_batch, workspace_bytes)
        self._bp, self._bwb, self._est = batch_params, batch_workspace_bytes, estimate_capacity
        self._gp, self._mp, self._wb = generate_pairs, make_params, workspace_bytes
        self._ap, self._ab, self._rb = allocate_pairs, allocate_batch, run_batch
        self._err, self._overflow = RhgError, OVERFLOW
        self.keep = keep_results

    def capacity(self, r: Request) -> int:
        return max(self._est(r.n, r.k), int(r.m_hint))

    def estimate(self, r: Request) -> int:
        return int(self._wb(self._mp(r.n, r.k, r.alpha, r.seed), 0)) + 8 * self.capacity(r)

    def estimate_batch(self, rs) -> int:
        return int(self._bwb(self._bp([(r.n, r.k, r.alpha, r.seed) for r in rs]))) + \
            8 * sum(self.capacity(r) for r in rs)

    def single(self, r: Request, stream):
        wsp = self._ap(self._mp(r.n, r.k, r.alpha, r.seed), self.capacity(r))
        try:
            pairs, res = self._gp(r.n, r.k, r.alpha, r.seed, workspace=wsp, stream=stream, overflow_retry=False)
        except self._err as e:
            if e.status == self._overflow and e.result is not None:
                return [Retry(int(e.result.m))]
            raise
        return [(int(res.m), float(res.R), pairs if self.keep else None)]

    def batch(self, rs, stream):
        params = self._bp([(r.n, r.k, r.alpha, r.seed) for r in rs])
        buf = self._ab(params, [self.capacity(r) for r in rs])
        rc, res, tot = self._rb(buf, stream)
        out = []
        for g, r in enumerate(rs):
            st = res[g].status
            if st == self._overflow:
                out.append(Retry(int(res[g].m)))
            elif st != 0:
                raise self._err(st, "rhg_generate_batch", tot)
            else:
                view = buf.out[2 * buf.offsets[g]: 2 * (buf.offsets[g] + res[g].m)].view(-1, 2)
                out.append((int(res[g].m), float(res[g].R), view if self.keep else None))
        return out


@dataclass
class _Work:
    reqs: list
    reserve: int


class Server:
    """budget_bytes: device memory the admitted requests may hold at once;
    workers: concurrent generations; small_n / batch_points: requests with
    n <= small_n are grouped, up to batch_points points per group."""

    def __init__(self, executor=None, budget_bytes: int = 120 * 10**9, workers: int = 4, small_n: int = 100_000,
                 batch_points: int = 4_000_000, batch_max: int = 256, use_cuda_streams: bool = True,
                 lookahead: int = 1024):
        self.ex = executor if executor is not None else GpuExecutor()
        self.budget = int(budget_bytes)
        self.free = int(budget_bytes)
        self.small_n, self.batch_points, self.batch_max = small_n, batch_points, batch_max
        self.lookahead = lookahead
        self.retries = 0
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
        """Admits the head of the queue (and small requests queued behind it) if it
        fits; else None."""
        head = self.queue[0]
        need = self.ex.estimate(head)
        if need > self.free:
            return None
        picked = [0]
        if head.n <= self.small_n:
            pts = head.n
            for i in range(1, min(len(self.queue), self.lookahead)):
                if len(picked) >= self.batch_max or pts >= self.batch_points:
                    break
                r = self.queue[i]
                if r.n <= self.small_n and pts + r.n <= self.batch_points:
                    picked.append(i)
                    pts += r.n
            if len(picked) > 1:
                reqs = [self.queue[i] for i in picked]
                need = self.ex.estimate_batch(reqs)
                while need > self.free and len(picked) > 1:
                    picked.pop()
                    reqs = [self.queue[i] for i in picked]
                    need = self.ex.estimate_batch(reqs) if len(picked) > 1 else self.ex.estimate(head)
                if need > self.free:
                    return None
        reqs = [self.queue[i] for i in picked]
        for i in reversed(picked):
            del self.queue[i]
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
                again = []
                for r, res in zip(work.reqs, out):
                    if isinstance(res, Retry):  # ran out of room: back to the head with its exact size
                        r.m_hint = max(int(res.m), r.m_hint + 1)
                        r.attempts += 1
                        again.append(r)
                        continue
                    m, R, pairs = res
                    self.done.append(Completion(r.rid, m, R, r.arrival, start, end, len(work.reqs), pairs))
                for r in reversed(again):
                    if self.ex.estimate(r) > self.budget:  # its exact size can never be admitted
                        self.errors.append(ValueError(f"request {r.rid} needs more than the budget {self.budget}"))
                        continue
                    self.queue.appendleft(r)
                self.retries += len(again)
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
