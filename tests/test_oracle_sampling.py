"""Pins for the oracle's points (Alg. 1 sampling step; Eq. 1) and bands
(Sec. III-A).  The radial coordinate is checked point by point against the
inverse-CDF identity F(r_i) = U_i, with F from Eq. 1 evaluated by numpy and U_i
from numpy's Philox, and in distribution by Kolmogorov-Smirnov tests."""
import math

import numpy as np
import pytest
from scipy import stats


def _u53(seed, n, word):
    out = np.empty(n, dtype=np.uint64)
    bg = np.random.Philox(counter=np.array([2**64 - 1] * 4, dtype=np.uint64),
                          key=np.array([seed, 0], dtype=np.uint64))
    raw = bg.random_raw(4 * n).reshape(n, 4)  # counters 0, 1, 2, ... in order
    out[:] = raw[:, word] >> np.uint64(11)
    return out


@pytest.mark.parametrize("n,k,alpha,seed", [(20000, 6, 1.0, 1), (20000, 16, 0.75, 2), (5000, 10, 0.55, 3),
                                            (5000, 10, 3.0, 4)])
def test_radius_inverse_cdf_pointwise(O, n, k, alpha, seed):
    R = O.target_radius(max(n, 1000), k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    U = _u53(seed, n, 1).astype(np.float64) * 2.0 ** -53
    F = np.expm1(alpha * r) ** 2 / (2 * np.exp(alpha * r)) / (math.cosh(alpha * R) - 1)  # (cosh ar - 1)/(cosh aR - 1)
    assert np.all(r >= 0) and np.all(r <= R)
    assert np.max(np.abs(F - U)) < 1e-9
    ph = _u53(seed, n, 0).astype(np.float64) * np.ldexp(2 * np.pi, -53)
    assert np.array_equal(ph, phi)


def test_distribution_ks(O):
    n, alpha = 200000, 0.8
    R = O.target_radius(10**6, 10, alpha)
    phi, r = O.sample_points(n, alpha, R, 77)
    assert stats.kstest(phi / (2 * np.pi), "uniform").pvalue > 1e-4
    F = (np.cosh(alpha * r) - 1) / (math.cosh(alpha * R) - 1)
    assert stats.kstest(F, "uniform").pvalue > 1e-4
    # a wrong exponent in the density is caught: the same r under alpha' = 0.9 is far off
    F_wrong = (np.cosh(0.9 * r) - 1) / (math.cosh(0.9 * R) - 1)
    assert stats.kstest(F_wrong, "uniform").pvalue < 1e-10


@pytest.mark.parametrize("B,p", [(1, 0.9), (2, 0.9), (14, 0.9), (24, 0.9), (20, 0.5), (10, 1.0), (8, 1.1)])
def test_boundaries(O, B, p):
    R = 23.5
    c = O.boundaries(R, B, p)
    assert c[0] == 0.0 and c[-1] == R and len(c) == B + 1
    w = np.diff(c)
    assert np.all(w > 0)
    if B >= 3:
        assert np.allclose(w[1:-1] / w[:-2], p, rtol=1e-12)
    # Sec. III-A: c_1 = (1-p) R / (1 - p^B) (equal widths when p = 1)
    c1 = R / B if p == 1.0 else (1 - p) * R / (1 - p**B)
    assert abs(c[1] - c1) <= 1e-12 * R if B > 1 else True
    assert abs(w.sum() - R) < 1e-12 * R


def test_default_bands(O):
    assert O.default_bands(2) == 1 and O.default_bands(3) == 2 and O.default_bands(4) == 2
    assert O.default_bands(10**4) == 14 and O.default_bands(10**6) == 20 and O.default_bands(10**7) == 24


def test_band_assignment(O):
    n, alpha = 50000, 1.0
    R = O.target_radius(n, 6, alpha)
    _, r = O.sample_points(n, alpha, R, 5)
    B = 16
    c = O.boundaries(R, B, 0.9)
    b = O.band_assign(r, R, B, 0.9)
    assert np.all(c[b] <= r)
    last = b == B - 1
    assert np.all(r[~last] < c[b[~last] + 1]) and np.all(r[last] <= R)
    assert np.array_equal(b, np.searchsorted(c[1:-1], r, side="right"))
