"""Rounding diagnostics of the device path against the oracle: the count of
examined pairs within the FP64 predicate's rounding band (|L - cosh R| <= 8 u
cosh r_v cosh r_w) and within 1e-12 of the threshold must be the oracle's exactly.
Every such pair is decided by the FP64 predicate on the device (the FP32 filter
and the core decide only pairs outside 32 u cosh r_v cosh r_w), and both sides'
windows admit all of them, so the counts are properties of the point set."""
import numpy as np
import pytest

from gpu_util import require_gpu, sorted_pairs
from planted import planted_pairs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("flags", [0, 1])
def test_planted_pairs_counts_equal_oracle(O, flags):
    """Pairs planted within 1e-12 .. 1e-6 of the threshold among random rim points,
    filter mode and FP64-only mode."""
    rhg = require_gpu()
    import torch
    phi_p, r_p, R = planted_pairs(npairs=240, seed=5)
    phi_s, r_s = O.sample_points(20_000, 1.0, R, 8)
    phi, r = np.concatenate([phi_s, phi_p]), np.concatenate([r_s, r_p])
    ref, st = O.band_edges(phi, r, R, O.default_bands(len(phi)), with_stats=True)
    pairs, res = rhg.edges_from_points(torch.from_numpy(phi).cuda(), torch.from_numpy(r).cuda(), R, flags=flags)
    assert np.array_equal(sorted_pairs(pairs), ref)
    assert st["rounding_band"] > 20
    assert res.rounding_band == st["rounding_band"]
    assert res.near_threshold == st["near_threshold"]


@pytest.mark.parametrize("n,k,alpha,seed", [(10_000, 6, 1.0, 1), (10**6, 16, 0.75, 2), (200_000, 2, 0.6, 7)])
def test_generated_graph_counts_equal_oracle(O, n, k, alpha, seed):
    rhg = require_gpu()
    _, res = rhg.generate_pairs(n, k, alpha, seed)
    R = O.target_radius(n, k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    m, _, st = O.band_count_subset(phi, r, R, O.default_bands(n), 0.9, np.arange(n, dtype=np.uint32),
                                   with_stats=True)
    assert res.m == m
    assert res.rounding_band == st["rounding_band"]
    assert res.near_threshold == st["near_threshold"]
