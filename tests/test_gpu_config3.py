"""Paper-scale graph (n = 10^7, k = 200, alpha = 1, seed 3; ~1G edges), in the
launch configuration bench.py times: exact edge count against the oracle's
Alg. 1 (OpenMP over all vertices), brute-force neighbourhoods of sampled
vertices (including the innermost hubs) and the global invariants."""
import numpy as np
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

N, K, ALPHA, SEED = 10**7, 200, 1.0, 3


@pytest.fixture(scope="module")
def gpu_graph():
    rhg = require_gpu()
    import torch
    pairs, res = rhg.generate_pairs(N, K, ALPHA, SEED)
    torch.cuda.synchronize()
    return pairs, res


@pytest.fixture(scope="module")
def oracle_points(O):
    R = O.target_radius(N, K, ALPHA)
    phi, r = O.sample_points(N, ALPHA, R, SEED)
    return R, phi, r


def test_invariants(gpu_graph):
    import torch
    pairs, res = gpu_graph
    assert pairs.shape == (res.m, 2)
    assert 0.9e9 < res.m < 1.2e9
    u = pairs[:, 0].to(torch.int64) & 0xFFFFFFFF
    v = pairs[:, 1].to(torch.int64) & 0xFFFFFFFF
    assert bool((u < v).all()) and int(v.max()) < N
    key = u * N + v
    del u, v
    key, _ = torch.sort(key)
    assert int((key[1:] == key[:-1]).sum()) == 0
    del key
    torch.cuda.empty_cache()


def test_edge_count_equals_oracle(O, gpu_graph, oracle_points):
    pairs, res = gpu_graph
    R, phi, r = oracle_points
    assert res.R == R
    m_ref, _ = O.band_count_subset(phi, r, R, O.default_bands(N), 0.9, np.arange(N, dtype=np.uint32))
    assert res.m == m_ref


def test_sampled_neighbourhoods(O, gpu_graph, oracle_points):
    import torch
    pairs, res = gpu_graph
    R, phi, r = oracle_points
    rng = np.random.default_rng(1)
    sample = np.unique(np.concatenate([rng.integers(0, N, 24), np.argsort(r)[:8], np.argsort(-r)[:4]]))
    s = torch.from_numpy(sample.astype(np.int64)).cuda()
    u = pairs[:, 0].to(torch.int64) & 0xFFFFFFFF
    v = pairs[:, 1].to(torch.int64) & 0xFFFFFFFF
    hit_u = torch.isin(u, s)
    hit_v = torch.isin(v, s)
    a = torch.cat([torch.stack([u[hit_u], v[hit_u]], 1), torch.stack([v[hit_v], u[hit_v]], 1)]).cpu().numpy()
    del u, v, hit_u, hit_v
    for vid in sample:
        got = np.sort(a[a[:, 0] == vid, 1])
        ref = O.neighbors(int(vid), phi, r, R).astype(np.int64)
        assert np.array_equal(got, ref), (vid, len(got), len(ref))
