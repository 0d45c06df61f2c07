"""Seeded input generator shared by the oracle and GPU tests: pairs of rim points
planted at a known exact distance from the threshold.  It computes inputs only
(positions from exact geometry in mpmath), never an expected edge set."""
import math

import numpy as np
import pytest


def planted_pairs(npairs=240, R=23.5, seed=5):
    """Pairs of rim points placed at angles whose exact L' = cosh(r_v - r_w) +
    2 sinh r_v sinh r_w sin^2(d/2) lies within +-1e-12 .. 1e-6 of cosh R relative
    (mpmath, 200 bits); the pairs sit 2 pi / npairs apart, so no other pair is near
    the threshold.  Returns (phi, r, R); pair j is points 2j and 2j + 1."""
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    rng = np.random.default_rng(seed)
    phi, r = [], []
    for j in range(npairs):
        a = 2 * math.pi * (j + 0.5) / npairs
        rv, rw = R - rng.uniform(0.2, 1.5), R - rng.uniform(0.2, 1.5)
        delta = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-12, -6)
        target = mp.cosh(mp.mpf(R)) * (1 + mp.mpf(delta))
        s2 = (target - mp.cosh(mp.mpf(rv) - mp.mpf(rw))) / (2 * mp.sinh(mp.mpf(rv)) * mp.sinh(mp.mpf(rw)))
        d = float(2 * mp.asin(mp.sqrt(s2)))
        phi += [a, a + d]
        r += [rv, rw]
    return np.array(phi), np.array(r), R
