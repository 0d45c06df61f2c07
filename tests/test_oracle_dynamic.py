"""Pins of the oracle's dynamic model (Sec. III-C, Algorithm 2, Theorem 1): the
movement against its closed forms in exact arithmetic (mpmath), reflection at
both boundaries, reversibility, and Theorem 1 (the positions keep their
distribution) by Kolmogorov-Smirnov tests that have the power to fail: small
disk, large steps, many iterated moves, and two negative controls (the sinh
coordinate that Algorithm 2 prints, and a wrong alpha), both of which must be
rejected."""
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


def _x(alpha, r):
    """The uniform radial coordinate cosh(alpha r) - 1, exactly."""
    return mp.cosh(mp.mpf(alpha) * mp.mpf(float(r))) - 1


def _sinh(alpha, r):
    return mp.sinh(mp.mpf(alpha) * mp.mpf(float(r)))


def test_rotation_and_radial_closed_forms(O):
    alpha, R = 0.8, 15.0
    rng = np.random.default_rng(5)
    n = 300
    phi = rng.uniform(0, 2 * np.pi, n)
    r = rng.uniform(5.0, 13.0, n)  # cosh(alpha r) - 1 in [26, 16400], top 81377: no reflection for |tau_r| <= 10
    tphi = rng.uniform(-1, 1, n)
    tr = rng.uniform(-10, 10, n)
    p2, r2, tr2 = O.move(np.arange(n), phi, r, tphi, tr, R, alpha)
    two_pi = mp.mpf(float.fromhex("0x1.921fb54442d18p+2"))
    for i in range(n):
        want = (mp.mpf(float(phi[i])) + mp.mpf(float(tphi[i]))) % two_pi
        assert 0.0 <= p2[i] < 2 * np.pi and abs(p2[i] - float(want)) <= 2.0 ** -50
        x_new = _x(alpha, r[i]) + mp.mpf(float(tr[i]))  # y = (cosh(alpha r) - 1) + tau_r
        assert abs(_x(alpha, r2[i]) / x_new - 1) < 1e-12
    assert np.array_equal(tr2, tr)  # no bounce, no sign change
    # the printed coordinate, kept for the negative control: y = sinh(alpha r) + tau_r
    p3, r3, _ = O.move(np.arange(n), phi, r, tphi, tr, R, alpha, coord=O.COORD_SINH)
    assert np.array_equal(p3, p2)
    for i in range(n):
        assert abs(_sinh(alpha, r3[i]) / (_sinh(alpha, r[i]) + mp.mpf(float(tr[i]))) - 1) < 1e-12


def test_small_radii_keep_their_precision(O):
    """Near the origin x = cosh(alpha r) - 1 ~ (alpha r)^2 / 2: it is evaluated as
    2 sinh^2(alpha r / 2) without cancellation (cosh(alpha r) - 1 in FP64 would
    lose all but ~4 digits of x at r = 1e-6), so a tiny step moves a tiny radius
    to within the deterministic asinh's absolute error of a few 2^-53."""
    alpha, R = 1.0, 10.0
    for r0, t in [(1e-6, 1e-13), (1e-4, 3e-9), (0.01, 1e-6)]:
        _, r2, _ = O.move([0], [1.0], [r0], [0.0], [t], R, alpha)
        want = float(mp.acosh(1 + _x(alpha, r0) + mp.mpf(t)) / alpha)
        assert abs(r2[0] - want) <= 1e-15 and abs(r2[0] - want) <= 1e-9 * want, (r0, r2[0], want)


def test_reflection_at_both_boundaries(O):
    alpha, R = 1.0, 10.0
    top = mp.cosh(mp.mpf(alpha) * mp.mpf(R)) - 1
    # near the rim, moving out by more than the distance to it
    r0 = float(mp.acosh(top - 49) / alpha)
    p2, r2, tr2 = O.move([0], [1.0], [r0], [0.0], [80.0], R, alpha)
    assert tr2[0] == -80.0 and r2[0] < R
    want = 2 * top - (_x(alpha, r0) + 80)
    assert abs(_x(alpha, r2[0]) / want - 1) < 1e-9
    # near the origin, moving in by more than the distance to it
    p2, r2, tr2 = O.move([0], [1.0], [0.001], [0.0], [-5.0], R, alpha)
    assert tr2[0] == 5.0
    assert abs(_x(alpha, r2[0]) - (5.0 - _x(alpha, 0.001))) < 1e-12
    # a point at the origin with an inward step bounces outward: x = 2
    p2, r2, tr2 = O.move([0], [3.0], [0.0], [0.0], [-2.0], R, alpha)
    assert tr2[0] == 2.0 and abs(r2[0] - math.acosh(3.0)) < 1e-15


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


# Theorem 1 on a small disk, where the coordinate matters: R = 3, alpha = 1, so
# cosh(alpha R) - 1 = 9.07 and sinh(alpha R) = 10.02; steps up to a quarter of the
# range, so every vertex crosses the disk many times in 80 steps.
SMALL_R, SMALL_ALPHA, SMALL_N, STEPS = 3.0, 1.0, 20_000, 80


def _iterate(O, move_alpha, coord, seed=31):
    phi, r = O.sample_points(SMALL_N, SMALL_ALPHA, SMALL_R, seed)
    top = math.cosh(SMALL_ALPHA * SMALL_R) - 1.0
    tphi, tr = O.draw_movement(SMALL_N, seed, (-1.0, 1.0), (-top / 4, top / 4))
    ids = np.arange(SMALL_N, dtype=np.uint32)
    for _ in range(STEPS):
        phi, r, tr = O.move(ids, phi, r, tphi, tr, SMALL_R, move_alpha, coord=coord)
    return phi, r


def _eq1_cdf(x):
    return (np.cosh(SMALL_ALPHA * x) - 1.0) / (np.cosh(SMALL_ALPHA * SMALL_R) - 1.0)


def test_theorem1_iterated_moves_keep_eq1(O):
    """80 moves of every vertex in the uniform coordinate: r still has the density
    of Eq. 1 and phi is still uniform; the sample has changed completely."""
    from scipy import stats
    phi0, r0 = O.sample_points(SMALL_N, SMALL_ALPHA, SMALL_R, 31)
    phi, r = _iterate(O, SMALL_ALPHA, O.COORD_UNIFORM)
    assert stats.kstest(r, _eq1_cdf).pvalue > 1e-3
    assert stats.kstest(phi / (2 * np.pi), "uniform").pvalue > 1e-3
    # the positions decorrelated from the start: the moved sample is a new draw
    assert abs(np.corrcoef(r, r0)[0, 1]) < 0.05


def test_theorem1_rejects_the_printed_sinh_coordinate(O):
    """Negative control: the same walk in sinh(alpha r), as Algorithm 2 prints it.
    Under Eq. 1 sinh(alpha r) has density x / ((cosh aR - 1) sqrt(1 + x^2)), not
    uniform, so the walk drifts towards the uniform law in sinh(alpha r), which
    puts too many vertices near the centre; the KS test must reject it."""
    from scipy import stats
    _, r = _iterate(O, SMALL_ALPHA, O.COORD_SINH)
    assert stats.kstest(r, _eq1_cdf).pvalue < 1e-8
    # and it converged to what a reflected walk converges to: uniform in sinh(alpha r)
    u = np.sinh(SMALL_ALPHA * r) / np.sinh(SMALL_ALPHA * SMALL_R)
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    assert np.mean(r < 1.0) > 1.5 * _eq1_cdf(1.0)


def test_theorem1_rejects_a_wrong_alpha(O):
    """Negative control: moving with alpha' = 1.4 on points drawn with alpha = 1
    maps to a coordinate that is not uniform for these points."""
    from scipy import stats
    _, r = _iterate(O, 1.4, O.COORD_UNIFORM)
    assert stats.kstest(r, _eq1_cdf).pvalue < 1e-8


def test_paper_experiment_step_keeps_the_distribution(O):
    """The paper's experiment (tau_phi in (-1, 1), tau_r in (-10, 1)) at a
    realistic radius, ten steps: phi uniform, r with the density of Eq. 1."""
    from scipy import stats
    n, alpha = 200_000, 1.0
    R = O.target_radius(n, 10, alpha)
    phi, r = O.sample_points(n, alpha, R, 21)
    tphi, tr = O.draw_movement(n, 21)
    ids = np.arange(n)
    p2, r2, tr2 = phi, r, tr
    for _ in range(10):
        p2, r2, tr2 = O.move(ids, p2, r2, tphi, tr2, R, alpha)
    cdf = lambda x: (np.cosh(alpha * x) - 1.0) / (np.cosh(alpha * R) - 1.0)
    assert stats.kstest(r2, cdf).pvalue > 1e-3
    assert stats.kstest(p2 / (2 * np.pi), "uniform").pvalue > 1e-3
    assert np.mean(p2 != phi) > 0.999 and np.mean(r2 != r) > 0.9
