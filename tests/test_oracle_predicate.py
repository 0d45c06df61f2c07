"""Pins for the oracle's edge predicate (Eq. 3 and the rule dist <= R of Alg. 1)
against the hyperbolic distance computed in another model: the Poincare disk,
in mpmath at 60 digits.  A wrong sign, a swapped cosh/sinh or a missing absolute
value in the oracle changes decisions far from the threshold and fails here."""
import math

import mpmath as mp
import numpy as np

mp.mp.dps = 60


def poincare_dist(ph1, r1, ph2, r2):
    z1 = mp.tanh(mp.mpf(r1) / 2) * mp.expj(mp.mpf(ph1))
    z2 = mp.tanh(mp.mpf(r2) / 2) * mp.expj(mp.mpf(ph2))
    return 2 * mp.atanh(abs(z1 - z2) / abs(1 - mp.conj(z1) * z2))


def test_predicate_vs_poincare(O):
    rng = np.random.default_rng(11)
    R = 16.7
    checked = 0
    for _ in range(1500):
        r1, r2 = rng.uniform(0, R, 2)
        ph1 = rng.uniform(0, 2 * math.pi)
        # bias towards small angular gaps so that both outcomes are common
        ph2 = (ph1 + rng.choice([-1, 1]) * rng.uniform(0, 1) ** 4 * math.pi) % (2 * math.pi)
        d = poincare_dist(ph1, r1, ph2, r2)
        L = O.edge_L(ph1, r1, ph2, r2)
        assert abs(mp.mpf(L) - mp.cosh(d)) <= 64 * 2.0**-53 * math.cosh(r1) * math.cosh(r2) + 1e-300
        if abs(d - R) > 1e-6:
            assert O.edge(ph1, r1, ph2, r2, R) == (d <= R)
            checked += 1
    assert checked > 1400


def test_special_cases(O):
    R = 12.0
    # equal angles: dist = |r1 - r2|
    assert O.edge(1.0, 3.0, 1.0, 3.0 + 11.9, R) and not O.edge(1.0, 0.5, 1.0, 0.5 + 12.1, R)
    # antipodal points: dist = r1 + r2
    assert O.edge(0.5, 5.9, 0.5 + math.pi, 6.0, R) and not O.edge(0.5, 6.1, 0.5 + math.pi, 6.0, R)
    # a point at the origin is adjacent to exactly the points with r <= R
    assert O.edge(0.0, 0.0, 2.0, 11.999, R) and not O.edge(0.0, 0.0, 2.0, 12.001, R)
    # symmetric
    rng = np.random.default_rng(3)
    for _ in range(200):
        a = rng.uniform(0, 2 * math.pi, 2)
        b = rng.uniform(0, R, 2)
        assert O.edge_L(a[0], b[0], a[1], b[1]) == O.edge_L(a[1], b[1], a[0], b[0])
