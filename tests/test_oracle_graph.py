"""Pins for the oracle's edge sets: the band algorithm (Alg. 1) against the all-pairs
definition on many small cases, band-count invariance, an all-pairs check in numpy
with the platform libm (agreement away from the threshold), the model's invariants
(symmetric set, no self-loops or duplicates) and its statistics: mean degree near k,
degree tail exponent near 2 alpha + 1 (Sec. II)."""
import math

import numpy as np
import pytest


def _check_pairs(pairs, n):
    assert pairs.ndim == 2 and pairs.shape[1] == 2
    if len(pairs):
        assert np.all(pairs[:, 0] < pairs[:, 1]) and pairs.max() < n
        key = pairs[:, 0].astype(np.uint64) * np.uint64(n) + pairs[:, 1]
        assert len(np.unique(key)) == len(pairs)


CASES = [(2, 0.5, 1.0, 1), (3, 1, 1.0, 2), (17, 4, 0.8, 3), (500, 6, 1.0, 4), (500, 30, 0.55, 5),
         (3000, 6, 1.0, 6), (3000, 12, 0.75, 7), (3000, 3, 3.0, 8), (2000, 60, 1.5, 9), (1000, 1, 1.0, 10)]


@pytest.mark.parametrize("n,k,alpha,seed", CASES)
def test_band_equals_brute(O, n, k, alpha, seed):
    R = O.target_radius(max(n, 2), k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    brute = O.brute_edges(phi, r, R)
    _check_pairs(brute, n)
    B0 = O.default_bands(n)
    for B, p in [(B0, 0.9), (1, 0.9), (2, 0.9), (min(64, 2 * B0), 0.9), (B0, 0.5), (B0, 1.0)]:
        band = O.band_edges(phi, r, R, B, p)
        assert np.array_equal(band, brute), (B, p)


def test_band_invariance_config1(O):
    g = O.generate(10**4, 6, 1.0, 1, with_stats=True)
    assert g["B"] == 14
    brute = O.brute_edges(g["phi"], g["r"], g["R"])
    assert np.array_equal(g["pairs"], brute)
    for B in (1, 7, 28, 64):
        assert np.array_equal(O.band_edges(g["phi"], g["r"], g["R"], B), brute)
    assert 5.0 < 2 * len(brute) / 1e4 < 7.5


def test_numpy_libm_all_pairs(O):
    """Same points, distances from numpy's libm in the well-conditioned form;
    every pair away from the threshold must be decided the same way."""
    n, k, alpha, seed = 4000, 8, 0.9, 12
    R = O.target_radius(n, k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    ours = O.band_edges(phi, r, R, O.default_bands(n))
    iu, ju = np.triu_indices(n, 1)
    d = np.abs(phi[iu] - phi[ju])
    L = np.cosh(r[iu] - r[ju]) + 2 * np.sinh(r[iu]) * np.sinh(r[ju]) * np.sin(d / 2) ** 2
    rel = (L - math.cosh(R)) / math.cosh(R)
    ref = rel <= 0
    clear = np.abs(rel) > 1e-9
    ours_mask = np.zeros(len(iu), dtype=bool)
    idx = {(int(a), int(b)) for a, b in ours}
    lin = np.array([a * n + b for a, b in idx], dtype=np.int64)
    ours_mask[np.isin(iu.astype(np.int64) * n + ju, lin)] = True
    assert np.array_equal(ours_mask[clear], ref[clear])
    assert (~clear).sum() < 5


@pytest.mark.slow
def test_statistics_config2(O):
    """Mean degree near k and a degree tail exponent near 2 alpha + 1 = 2.5."""
    n, k, alpha = 10**6, 16, 0.75
    g = O.generate(n, k, alpha, 2, with_stats=True)
    pairs = g["pairs"]
    _check_pairs(pairs, n)
    deg = np.bincount(pairs.ravel(), minlength=n)
    assert abs(deg.mean() / k - 1) < 0.05
    # discrete power-law MLE (Clauset, Shalizi, Newman 2009, Eq. 3.7 approximation)
    kmin = 50
    tail = deg[deg >= kmin].astype(np.float64)
    gamma = 1 + len(tail) / np.sum(np.log(tail / (kmin - 0.5)))
    assert abs(gamma - (2 * alpha + 1)) < 0.35, gamma
    assert g["stats"]["candidates"] >= len(pairs)
    assert g["stats"]["candidates"] < 3 * len(pairs)


def test_timed_baseline_counts_the_outward_edges(O):
    """The timed CPU baseline (band structure built once, outward queries of a
    vertex set) counts each edge from its outward endpoint: over all vertices it
    gives the all-pairs edge count, on one thread and on all threads alike."""
    n, k, alpha, seed = 3000, 12, 0.75, 7
    R = O.target_radius(n, k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    m = len(O.brute_edges(phi, r, R))
    prep = O.Prepared(phi, r, R, O.default_bands(n), 0.9)
    try:
        ids = np.arange(n, dtype=np.uint32)
        m_all, threads = prep.count_edges(ids)
        m_one, one = prep.count_edges(ids, threads=1)
        assert m_all == m_one == m
        assert one == 1 and threads == O.openmp_threads()
        halves = prep.count_edges(ids[: n // 2])[0] + prep.count_edges(ids[n // 2:])[0]
        assert halves == m
    finally:
        prep.close()
