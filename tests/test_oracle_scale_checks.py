"""Pins of the oracle's checks for large graphs.

- The ordered edge emitter (every edge (u, w), u < w, of a vertex range, by a
  windowed search of all bands) equals the all-pairs definition on small cases,
  in any cut into ranges, and equals Alg. 1 on a medium graph; the GPU's
  paper-scale graph is compared with it pair by pair.
- The window check (Sec. III-B getMinMaxPhi): every all-pairs edge of sampled
  vertices lies inside the window of its band (0 misses) at n = 10^6 (and at
  n = 10^7 in the slow set); windows narrowed by 1 % are caught.
- The rounding diagnostics (pairs inside the FP64 predicate's rounding band,
  pairs the cancellation-free form decides otherwise) on planted pairs whose
  exact distance is known from mpmath.
"""
import math

import numpy as np
import pytest

from planted import planted_pairs as _planted_pairs

CASES = [(2, 0.5, 1.0, 1), (17, 4, 0.8, 3), (500, 6, 1.0, 4), (500, 30, 0.55, 5), (3000, 6, 1.0, 6),
         (3000, 3, 3.0, 8), (2000, 60, 1.5, 9), (1000, 1, 1.0, 10)]


@pytest.mark.parametrize("n,k,alpha,seed", CASES)
def test_upper_pairs_equal_all_pairs(O, n, k, alpha, seed):
    R = O.target_radius(max(n, 2), k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    brute = O.brute_edges(phi, r, R)
    B0 = O.default_bands(n)
    for B in (1, B0, min(64, 2 * B0)):
        prep = O.Prepared(phi, r, R, B, 0.9)
        try:
            assert np.array_equal(prep.upper_pairs(0, n), brute), B
            cuts = sorted({0, n, n // 3, n // 2, (2 * n) // 3})
            parts = [prep.upper_pairs(a, b) for a, b in zip(cuts[:-1], cuts[1:])]
            assert np.array_equal(np.concatenate(parts), brute), B
        finally:
            prep.close()


def test_upper_pairs_equal_alg1_medium(O):
    n, k, alpha, seed = 200_000, 20, 0.8, 17
    R = O.target_radius(n, k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    B = O.default_bands(n)
    alg1 = O.band_edges(phi, r, R, B)
    prep = O.Prepared(phi, r, R, B, 0.9)
    try:
        got = np.concatenate([prep.upper_pairs(a, min(a + 65536, n)) for a in range(0, n, 65536)])
    finally:
        prep.close()
    assert np.array_equal(got, alg1)


def _window_check(O, n, k, alpha, seed, nsample, ninner, slow=False):
    R = O.target_radius(n, k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    rng = np.random.default_rng(seed)
    ids = np.unique(np.concatenate([rng.integers(0, n, nsample), np.argsort(r)[:ninner]])).astype(np.uint32)
    prep = O.Prepared(phi, r, R, O.default_bands(n), 0.9)
    try:
        res = prep.window_misses(ids)
        narrow = prep.window_misses(ids, theta_scale=0.99)
    finally:
        prep.close()
    return res, narrow


def test_window_misses_config2(O):
    """n = 10^6, k = 16, alpha = 0.75 (the CSR workload): 300 random vertices and
    the 12 innermost (hubs whose windows span whole bands)."""
    res, narrow = _window_check(O, 10**6, 16, 0.75, 2, 300, 12)
    assert res["edges"] > 300 * 16
    assert res["misses"] == 0
    # Alg. 1 from these vertices finds exactly the edges they are the inner endpoint of
    assert res["alg1_edges"] == res["inner_endpoint_edges"]
    # the check has power: windows 1 % too narrow lose edges
    assert narrow["misses"] > 0


@pytest.mark.slow
def test_window_misses_config3(O):
    """n = 10^7, k = 200, alpha = 1 (the paper-scale workload): 40 random vertices
    and the 8 innermost hubs, every one of their ~10^4 all-pairs edges inside its
    window."""
    res, narrow = _window_check(O, 10**7, 200, 1.0, 3, 40, 8)
    assert res["edges"] > 40 * 100
    assert res["misses"] == 0
    assert res["alg1_edges"] == res["inner_endpoint_edges"]
    assert narrow["misses"] > 0


def test_rounding_diagnostics_on_planted_pairs(O):
    """The canonical predicate (Eq. 3 as a fixed FP64 sequence) against exact
    geometry on pairs planted within its rounding noise: the oracle's counters
    must equal the counts taken from mpmath and from the canonical values."""
    mp = pytest.importorskip("mpmath")
    phi, r, R = _planted_pairs()
    coshR = float(O.dm("cosh", [R])[0])
    ch = O.dm("cosh", r)
    exact_wrong = band = near = 0
    canon_edges = []
    for j in range(0, len(phi), 2):
        v, w = j, j + 1
        L = O.edge_L(phi[v], r[v], phi[w], r[w])
        canon = L <= coshR
        dd = abs(mp.mpf(phi[v]) - mp.mpf(phi[w]))
        Lx = mp.cosh(mp.mpf(r[v]) - mp.mpf(r[w])) + 2 * mp.sinh(mp.mpf(r[v])) * mp.sinh(mp.mpf(r[w])) * mp.sin(dd / 2) ** 2
        exact = Lx <= mp.cosh(mp.mpf(R))
        exact_wrong += canon != exact
        band += abs(L - coshR) <= 2.0 ** -50 * (ch[v] * ch[w])
        near += abs(L - coshR) <= 1e-12 * coshR
        if canon:
            canon_edges.append((v, w))
    # the planted set must exercise the counters
    assert exact_wrong >= 10 and band >= exact_wrong
    for B in (O.default_bands(len(phi)), 1):
        pairs, st = O.band_edges(phi, r, R, B, with_stats=True)
        assert [tuple(p) for p in pairs] == canon_edges
        assert st["rounding_band"] == band
        assert st["near_threshold"] == near
        assert st["disagree_longdouble_wellcond"] == exact_wrong
        assert st["disagree_fp64_wellcond"] == exact_wrong


def test_rounding_band_is_band_count_invariant(O):
    """Windows only prune: every pair within the rounding band is examined for any
    band count (B = 1 examines all pairs).  Planted pairs inside a random point
    set of the same disk."""
    phi_p, r_p, R = _planted_pairs(npairs=120, seed=9)
    phi_s, r_s = O.sample_points(4000, 1.0, R, 8)
    phi, r = np.concatenate([phi_s, phi_p]), np.concatenate([r_s, r_p])
    ref = None
    for B in (1, O.default_bands(len(phi)), 40):
        pairs, st = O.band_edges(phi, r, R, B, with_stats=True)
        got = (len(pairs), st["rounding_band"], st["near_threshold"], st["disagree_fp64_wellcond"],
               st["disagree_longdouble_wellcond"])
        ref = ref or got
        assert got == ref
    assert ref[1] > 0 and ref[3] > 0
