"""The FP32 filter decides only pairs its error bound makes certain: with
RHG_FLAG_VERIFY every decided pair is also evaluated with the FP64 predicate
(Eq. 3) and any contradiction is counted.  Edge sets in filter mode, FP64 mode
and the oracle agree."""
import numpy as np
import pytest

from gpu_util import require_gpu, sorted_pairs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,k,alpha,seed", [(10_000, 6, 1.0, 1), (200_000, 16, 0.75, 2), (300_000, 60, 1.0, 5),
                                            (100_000, 8, 0.6, 7), (50_000, 10, 2.5, 8)])
def test_filter_decisions_verified(O, n, k, alpha, seed):
    rhg = require_gpu()
    pairs, res = rhg.generate_pairs(n, k, alpha, seed, flags=rhg.FLAG_VERIFY)
    assert res.mode == 1
    assert res.verify_failures == 0
    fp64, res64 = rhg.generate_pairs(n, k, alpha, seed, flags=rhg.FLAG_FP64_ONLY)
    assert res64.mode == 0
    assert np.array_equal(sorted_pairs(pairs), sorted_pairs(fp64))
    assert res.near_threshold == res64.near_threshold
    assert res.rechecks < 0.01 * res.candidates


def test_config3_filter_verified():
    """Every decided pair of n = 10^7, k = 200 checked against the FP64 predicate."""
    rhg = require_gpu()
    _, res = rhg.generate_pairs(10**7, 200, 1.0, 3, flags=rhg.FLAG_VERIFY)
    assert res.mode == 1 and res.verify_failures == 0
    assert 0.9e9 < res.m < 1.2e9


def test_large_R_uses_fp64_mode(O):
    """R > 32: the FP64 noise of Eq. 3 exceeds any useful FP32 margin; FP64 mode."""
    rhg = require_gpu()
    n, k, alpha, seed = 10**6, 1, 0.6, 3
    pairs, res = rhg.generate_pairs(n, k, alpha, seed)
    assert res.R > 32 and res.mode == 0
    R = O.target_radius(n, k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    ref = O.band_edges(phi, r, R, O.default_bands(n))
    assert np.array_equal(sorted_pairs(pairs), ref)


def test_seam_pairs_verified(O):
    """Points on both sides of the 0 / 2 pi seam near the rim: the filter's angular
    distance must stay accurate when it wraps (FP32 2 pi - |d| would not)."""
    rhg = require_gpu()
    import math
    import torch
    rng = np.random.default_rng(21)
    n, R = 6000, 20.0
    phi = np.concatenate([rng.uniform(0, 3e-4, n // 2), np.nextafter(2 * math.pi, 0) - rng.uniform(0, 3e-4, n // 2)])
    r = rng.uniform(R - 3, R, n)
    pairs, res = rhg.edges_from_points(torch.from_numpy(phi).cuda(), torch.from_numpy(r).cuda(), R,
                                       flags=rhg.FLAG_VERIFY)
    assert res.mode == 1 and res.verify_failures == 0
    assert np.array_equal(sorted_pairs(pairs), O.brute_edges(phi, r, R))


@pytest.mark.parametrize("n,k,alpha,seed", [(5 * 10**6, 8, 0.6, 21), (2 * 10**6, 4, 0.55, 22)])
def test_solved_R_above_filter_range_runs_fp64_mode(O, n, k, alpha, seed):
    """Graphs whose R solved from Eq. 22 is above 32 run in FP64 mode; the host
    sizes their chunk list for it (no RHG_ERR_OOM) and the edge count is the
    oracle's Alg. 1 count."""
    rhg = require_gpu()
    _, res = rhg.generate_pairs(n, k, alpha, seed)
    R = O.target_radius(n, k, alpha)
    assert R > 32 and res.R == R and res.mode == 0
    phi, r = O.sample_points(n, alpha, R, seed)
    m, _ = O.band_count_subset(phi, r, R, O.default_bands(n), 0.9, np.arange(n, dtype=np.uint32))
    assert res.m == m
