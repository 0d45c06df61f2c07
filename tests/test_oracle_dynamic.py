"""Pins of the oracle's dynamic model (Sec. III-C, Algorithm 2): the movement
against its closed forms in exact arithmetic (mpmath), reflection at both
boundaries, reversibility, and the paper's Theorem 1 (the positions keep their
distribution) by Kolmogorov-Smirnov tests."""
import math

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
mp.mp.prec = 200


def test_asinh_against_mpmath(O):
    rng = np.random.default_rng(3)
    ys = np.concatenate([10.0 ** rng.uniform(-6, 35, 400), [0.0, 1.0, 2.0, 1e-300, 5e30]])
    for y in ys:
        exact = float(mp.asinh(mp.mpf(float(y))))
        got = O.asinh(float(y))
        if y >= 1.0:
            assert abs(got - exact) <= 4 * math.ulp(exact), y
        else:  # the log form keeps an absolute error of a few 2^-53 near 0
            assert abs(got - exact) <= 2.0 ** -51, y


def test_draw_movement_ranges_and_uniformity(O):
    from scipy import stats
    tphi, tr = O.draw_movement(200_000, 9)
    assert tphi.min() >= -1.0 and tphi.max() < 1.0 and tr.min() >= -10.0 and tr.max() < 1.0
    assert stats.kstest((tphi + 1.0) / 2.0, "uniform").pvalue > 1e-3
    assert stats.kstest((tr + 10.0) / 11.0, "uniform").pvalue > 1e-3
    a, b = O.draw_movement(1000, 9, (0.5, 0.5), (2.0, 2.0))
    assert np.all(a == 0.5) and np.all(b == 2.0)


def _sinh(alpha, r):
    return mp.sinh(mp.mpf(alpha) * mp.mpf(float(r)))


def test_rotation_and_radial_closed_forms(O):
    alpha, R = 0.8, 15.0
    rng = np.random.default_rng(5)
    n = 300
    phi = rng.uniform(0, 2 * np.pi, n)
    r = rng.uniform(5.0, 13.0, n)  # sinh(alpha r) in [27, 16400], top 81377: no reflection for |tau_r| <= 10
    tphi = rng.uniform(-1, 1, n)
    tr = rng.uniform(-10, 10, n)
    p2, r2, tr2 = O.move(np.arange(n), phi, r, tphi, tr, R, alpha)
    two_pi = mp.mpf(float.fromhex("0x1.921fb54442d18p+2"))
    for i in range(n):
        want = (mp.mpf(float(phi[i])) + mp.mpf(float(tphi[i]))) % two_pi
        assert 0.0 <= p2[i] < 2 * np.pi and abs(p2[i] - float(want)) <= 2.0 ** -50
        x_new = _sinh(alpha, r[i]) + mp.mpf(float(tr[i]))  # Algorithm 2: y = sinh(alpha r) + tau_r
        assert abs(_sinh(alpha, r2[i]) / x_new - 1) < 1e-12
    assert np.array_equal(tr2, tr)  # no bounce, no sign change


def test_reflection_at_both_boundaries(O):
    alpha, R = 1.0, 10.0
    top = mp.sinh(mp.mpf(alpha) * mp.mpf(R))
    # near the rim, moving out by more than the distance to it
    r0 = float(mp.asinh(top - 50) / alpha)
    p2, r2, tr2 = O.move([0], [1.0], [r0], [0.0], [80.0], R, alpha)
    assert tr2[0] == -80.0 and r2[0] < R
    want = 2 * top - (_sinh(alpha, r0) + 80)
    assert abs(_sinh(alpha, r2[0]) / want - 1) < 1e-9
    # near the origin, moving in by more than the distance to it
    p2, r2, tr2 = O.move([0], [1.0], [0.001], [0.0], [-5.0], R, alpha)
    assert tr2[0] == 5.0
    assert abs(_sinh(alpha, r2[0]) - (5.0 - _sinh(alpha, 0.001))) < 1e-12
    # a point at the origin with an inward step bounces outward
    p2, r2, tr2 = O.move([0], [3.0], [0.0], [0.0], [-2.0], R, alpha)
    assert tr2[0] == 2.0 and abs(r2[0] - math.asinh(2.0)) < 1e-15


def test_only_listed_nodes_move_and_steps_invert(O):
    alpha, R = 1.0, 16.0
    phi, r = O.sample_points(1000, alpha, R, 4)
    tphi, tr = O.draw_movement(1000, 4)
    ids = np.arange(0, 1000, 3)
    p2, r2, tr2 = O.move(ids, phi, r, tphi, tr, R, alpha)
    still = np.setdiff1d(np.arange(1000), ids)
    assert np.array_equal(p2[still], phi[still]) and np.array_equal(r2[still], r[still])
    assert np.all(p2[ids] != phi[ids])
    # back with the negated steps: where no bounce happened the positions return
    p3, r3, _ = O.move(ids, p2, r2, -tphi, -tr2, R, alpha)
    ok = tr2[ids] == tr[ids]
    assert ok.mean() > 0.9
    dphi = np.abs(p3[ids] - phi[ids])
    dphi = np.minimum(dphi, 2 * np.pi - dphi)
    assert np.all(dphi < 1e-12)
    assert np.all(np.abs(r3[ids][ok] - r[ids][ok]) < 1e-9)


def test_movement_preserves_the_point_distribution(O):
    """Theorem 1: after a movement step of every node (the paper's experiment:
    tau_phi in (-1, 1), tau_r in (-10, 1)) phi stays uniform and r keeps the
    density alpha sinh(alpha r) / (cosh(alpha R) - 1)."""
    from scipy import stats
    n, alpha = 200_000, 1.0
    R = O.target_radius(n, 10, alpha)
    phi, r = O.sample_points(n, alpha, R, 21)
    tphi, tr = O.draw_movement(n, 21)
    p2, r2, _ = O.move(np.arange(n), phi, r, tphi, tr, R, alpha)
    cdf = lambda x: (np.cosh(alpha * x) - 1.0) / (np.cosh(alpha * R) - 1.0)
    assert stats.kstest(r2, cdf).pvalue > 1e-3
    assert stats.kstest(p2 / (2 * np.pi), "uniform").pvalue > 1e-3
    # and the moved positions really changed
    assert np.mean(p2 != phi) > 0.999 and np.mean(r2 != r) > 0.9
