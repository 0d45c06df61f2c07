"""Pins for the oracle's R (Sec. III-B getTargetRadius, Eq. 22 of Krioukov et al.).

Independent reference: the exact expected degree of the threshold model, i.e.
(n-1) times the probability that two independent points (radial density Eq. 1,
uniform angle) lie within distance R, by adaptive quadrature in scipy.  Eq. 22 is
an approximation of that quantity; at the sizes below it agrees to 1e-3 or better,
so a dropped or mis-signed term in the oracle's Eq. 22 fails the test."""
import math

import numpy as np
import pytest
from scipy import integrate


def k_exact(n, alpha, R):
    C = math.cosh(alpha * R) - 1.0
    chR = math.cosh(R)

    def f(r):
        return alpha * math.sinh(alpha * r) / C

    def theta(r1, r2):
        if r1 + r2 <= R:
            return math.pi
        q = (chR - math.cosh(r1 - r2)) / (2 * math.sinh(r1) * math.sinh(r2))
        if q <= 0:
            return 0.0
        if q >= 1:
            return math.pi
        return 2 * math.asin(math.sqrt(q))

    def inner(r1):
        return integrate.quad(lambda r2: f(r2) * theta(r1, r2) / math.pi, 0, R,
                              points=[max(0.0, R - r1)], limit=200, epsabs=0, epsrel=1e-10)[0]

    val = integrate.quad(lambda r1: f(r1) * inner(r1), 0, R, limit=200, epsabs=0, epsrel=1e-9)[0]
    return (n - 1) * val


@pytest.mark.parametrize("n,k,alpha,tol", [
    (10**6, 16, 0.75, 1e-3),
    (10**7, 200, 1.0, 1e-3),
    (10**6, 8, 0.6, 5e-3),
    (10**5, 10, 2.0, 1e-3),
])
def test_radius_gives_exact_expected_degree(O, n, k, alpha, tol):
    R = O.target_radius(n, k, alpha)
    assert abs(k_exact(n, alpha, R) / k - 1) < tol


@pytest.mark.parametrize("n,k,alpha,R_expected", [
    (10**4, 6, 1.0, 16.705), (10**6, 16, 0.75, 25.564), (10**7, 200, 1.0, 23.509)])
def test_radius_config_values(O, n, k, alpha, R_expected):
    # the three plain configurations: independent numpy estimates to ~1e-3
    assert abs(O.target_radius(n, k, alpha) - R_expected) < 2e-3


def test_radius_asymptotic_form(O):
    # for large n the e^{-R/2} term dominates: R ~ 2 ln(2 xi^2 n / (pi k))  (cf. R = 2 ln n + C)
    for n, k, alpha in [(10**7, 10, 1.0), (10**8, 20, 1.5), (10**9, 50, 1.0)]:
        xi = alpha / (alpha - 0.5)
        R_asym = 2 * math.log(2 * xi * xi * n / (math.pi * k))
        assert abs(O.target_radius(n, k, alpha) - R_asym) < 2e-3


def test_bisection_brackets_adjacent_doubles(O):
    for n, k, alpha in [(10**4, 6, 1.0), (10**6, 16, 0.75), (10**7, 200, 1.0), (1000, 30, 0.55)]:
        R = O.target_radius(n, k, alpha)
        below = np.nextafter(R, 0.0)
        assert O.kbar(R, n, alpha) <= k < O.kbar(below, n, alpha)


def test_radius_monotone(O):
    Rs = [O.target_radius(10**5, k, 1.0) for k in (2, 4, 8, 16, 32)]
    assert all(a > b for a, b in zip(Rs, Rs[1:]))
    Rs = [O.target_radius(n, 8, 1.0) for n in (10**3, 10**4, 10**5, 10**6)]
    assert all(a < b for a, b in zip(Rs, Rs[1:]))


def test_radius_errors(O):
    assert O.target_radius_status(1, 6, 1.0)[0] == O.STATUS_INVALID_ARG
    assert O.target_radius_status(1000, 6, 0.5)[0] == O.STATUS_INVALID_ARG
    assert O.target_radius_status(1000, 0.0, 1.0)[0] == O.STATUS_INVALID_ARG
    assert O.target_radius_status(1000, -1.0, 1.0)[0] == O.STATUS_INVALID_ARG
    assert O.target_radius_status(2**32, 6, 1.0)[0] == O.STATUS_INVALID_ARG
    # a denser graph than the approximation can express
    assert O.target_radius_status(100, 1e6, 1.0)[0] == O.STATUS_NO_SOLUTION
