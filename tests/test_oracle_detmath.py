"""Pins for the oracle's deterministic FP64 elementary functions: exact checks of
their constants against mpmath, and error bounds against mpmath at high precision.
A dropped Taylor term, a wrong sign or a bad reduction constant breaks the bounds."""
import math

import mpmath as mp
import numpy as np
import pytest

mp.mp.prec = 200
U = 2.0 ** -53


def _ulp_err(got, exact):
    exact = mp.mpf(exact)
    if exact == 0:
        return abs(mp.mpf(got)) / mp.mpf(2.0 ** -1074)
    ulp = mp.mpf(2) ** (mp.floor(mp.log(abs(exact), 2)) - 52)
    return float(abs(mp.mpf(got) - exact) / ulp)


def test_constants(O):
    c = O.constants()
    pi, ln2 = mp.pi, mp.log(2)
    assert c["PI"] == float(pi) and c["TWO_PI"] == 2 * c["PI"]
    assert c["INV_LN2"] == float(1 / ln2) and c["TWO_OVER_PI"] == float(2 / pi)
    assert c["SQRT_HALF"] == float(mp.sqrt(mp.mpf(0.5)))
    # split ln 2: HI has at most 32 significant bits, HI + LO = ln 2 to ~2^-85
    m, e = math.frexp(c["LN2_HI"])
    assert (m * 2**32) == int(m * 2**32)
    assert abs(mp.mpf(c["LN2_HI"]) + mp.mpf(c["LN2_LO"]) - ln2) < mp.mpf(2) ** -85
    # three-part pi/2: first two parts at most 33 significant bits
    for k in ("PIO2_1", "PIO2_2"):
        m, e = math.frexp(c[k])
        assert m * 2**33 == int(m * 2**33)
    s = mp.mpf(c["PIO2_1"]) + mp.mpf(c["PIO2_2"]) + mp.mpf(c["PIO2_3"])
    assert abs(s - pi / 2) < mp.mpf(2) ** -120


def _sweep(lo, hi, n, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(lo, hi, n), np.linspace(lo, hi, 257)])


def test_exp(O):
    xs = np.concatenate([_sweep(-60, 60, 1500, 1), [0.0, 1.0, -1.0, 0.3465, -0.3466, 708.0, 1e-300]])
    got = O.dm("exp", xs)
    worst = max(_ulp_err(g, mp.exp(mp.mpf(x))) for g, x in zip(got, xs))
    assert worst <= 1.5, worst
    assert O.dm("exp", [0.0])[0] == 1.0


def test_log(O):
    rng = np.random.default_rng(2)
    xs = np.concatenate([np.exp(rng.uniform(-40, 60, 1500)), 1 + rng.uniform(-1e-3, 1e-3, 300),
                         1 + rng.uniform(-1e-12, 1e-12, 50), [1.0, 2.0, 0.5, 0.7071067811865476,
                                                              1.4142135623730951, 1e300, 1e-300]])
    got = O.dm("log", xs)
    worst = max(_ulp_err(g, mp.log(mp.mpf(x))) for g, x in zip(got, xs) if x != 1.0)
    assert worst <= 2.0, worst
    assert O.dm("log", [1.0])[0] == 0.0


def test_cos(O):
    xs = np.concatenate([_sweep(0, 2 * math.pi, 3000, 3), [0.0, math.pi / 2, math.pi,
                                                           3 * math.pi / 2, 2 * math.pi, 1e-9]])
    got = O.dm("cos", xs)
    abs_err = max(abs(mp.mpf(g) - mp.cos(mp.mpf(x))) for g, x in zip(got, xs))
    assert abs_err <= 2 * U, abs_err / U
    big = [(g, x) for g, x in zip(got, xs) if abs(math.cos(x)) > 0.25]
    worst = max(_ulp_err(g, mp.cos(mp.mpf(x))) for g, x in big)
    assert worst <= 2.0, worst
    assert O.dm("cos", [0.0])[0] == 1.0


@pytest.mark.parametrize("fn", ["cosh", "sinh"])
def test_cosh_sinh(O, fn):
    xs = np.concatenate([_sweep(0, 60, 1500, 4), _sweep(0, 0.6, 500, 5), [0.0, 0.5, 0.4999999, 1e-8]])
    got = O.dm(fn, xs)
    ref = mp.cosh if fn == "cosh" else mp.sinh
    worst = max(_ulp_err(g, ref(mp.mpf(x))) for g, x in zip(got, xs) if x > 0 or fn == "cosh")
    assert worst <= 2.5, worst


def test_monotone_on_path_domain(O):
    # r -> cosh r and sinh r feed the predicate; check they do not decrease on a fine grid
    xs = np.linspace(0, 30, 20001)
    for fn in ("cosh", "sinh", "exp"):
        v = O.dm(fn, xs)
        assert np.all(np.diff(v) >= 0), fn
