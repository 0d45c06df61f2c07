"""Paper-scale graph (n = 10^7, k = 200, alpha = 1, seed 3; ~1G edges), in the
launch configuration bench.py times, compared with the oracle pair by pair: the
device pairs are sorted on the device by (u, v) and compared element by element
with the oracle's ordered edge list (every edge (u, w), u < w, of a vertex range
from a windowed search of all bands), one vertex range at a time, over all
~10^9 pairs.  Also the exact edge count and rounding diagnostics of the oracle's
Alg. 1 and the global invariants."""
import numpy as np
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

N, K, ALPHA, SEED = 10**7, 200, 1.0, 3
RANGE = 1 << 19  # vertices per compared range (~5e7 pairs)


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


def test_edge_count_and_diagnostics_equal_oracle(O, gpu_graph, oracle_points):
    pairs, res = gpu_graph
    R, phi, r = oracle_points
    assert res.R == R
    m_ref, _, st = O.band_count_subset(phi, r, R, O.default_bands(N), 0.9, np.arange(N, dtype=np.uint32),
                                       with_stats=True)
    assert res.m == m_ref
    assert res.rounding_band == st["rounding_band"]
    assert res.near_threshold == st["near_threshold"]


def test_every_pair_equals_oracle(O, gpu_graph, oracle_points):
    """All ~10^9 pairs, element by element, in ranges of 2^19 vertices."""
    import torch
    pairs, res = gpu_graph
    R, phi, r = oracle_points
    key = ((pairs[:, 0].to(torch.int64) & 0xFFFFFFFF) << 32) | (pairs[:, 1].to(torch.int64) & 0xFFFFFFFF)
    key, _ = torch.sort(key)
    bounds = torch.arange(0, N + RANGE, RANGE, dtype=torch.int64, device=key.device).clamp(max=N) << 32
    at = torch.searchsorted(key, bounds).cpu().numpy()
    prep = O.Prepared(phi, r, R, O.default_bands(N), 0.9)
    compared = 0
    try:
        for j, u0 in enumerate(range(0, N, RANGE)):
            u1 = min(u0 + RANGE, N)
            got = key[at[j]:at[j + 1]].cpu().numpy()
            ref = prep.upper_pairs(u0, u1, capacity=int(len(got) * 1.1) + 4096)
            ref_key = (ref[:, 0].astype(np.int64) << 32) | ref[:, 1].astype(np.int64)
            assert len(got) == len(ref_key), (u0, len(got), len(ref_key))
            bad = np.flatnonzero(got != ref_key)
            assert len(bad) == 0, (u0, [(int(got[b] >> 32), int(got[b] & 0xFFFFFFFF)) for b in bad[:4]])
            compared += len(got)
    finally:
        prep.close()
        del key
        torch.cuda.empty_cache()
    assert compared == res.m
