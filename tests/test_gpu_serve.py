"""Served generation on the GPU: requests generated concurrently (overlapping
streams, small ones grouped into batches) give each the same edge set as the
same request generated alone."""
import numpy as np
import pytest

from gpu_util import require_gpu, sorted_pairs

pytestmark = pytest.mark.gpu


def test_each_result_same_alone_and_in_the_mix():
    rhg = require_gpu()
    from paper_1606_09481_gb300.serve import GpuExecutor, Request, Server
    rng = np.random.default_rng(11)
    reqs = [Request(j, int(10 ** rng.uniform(3.3, 5.3)), int(rng.integers(8, 41)), float(rng.uniform(0.6, 1.2)),
                    10**6 + j, 0.0) for j in range(24)]
    srv = Server(GpuExecutor(keep_results=True), budget_bytes=8 * 10**9, workers=3, small_n=30_000,
                 batch_points=150_000)
    for r in reqs:
        srv.submit(r)
    srv.close()
    done = sorted(srv.done, key=lambda c: c.rid)
    assert [c.rid for c in done] == list(range(24))
    assert max(c.batch_size for c in done) > 1  # some requests ran in a batch
    for r, c in zip(reqs, done):
        pairs, res = rhg.generate_pairs(r.n, r.k, r.alpha, r.seed)
        assert c.m == res.m and c.R == res.R
        assert np.array_equal(sorted_pairs(c.pairs), sorted_pairs(pairs)), r.rid
