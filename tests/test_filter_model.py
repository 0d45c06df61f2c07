"""The FP32 filter's error model, checked on the CPU.

The device decides a candidate pair in FP32 (X = P_v M_w + M_v P_w +
2 S_v S_w sin^2(d/2), which is Eq. 3 divided by cosh R) only when |X - 1|
exceeds its error bound; every other pair goes to the FP64 predicate.  This
test restates that arithmetic in numpy float32, operation by operation
(filter values as the gather stores them, then the decision), perturbs the
radius by the largest error of the FP32-assisted sampler radius, and checks on
adversarial pairs right at the threshold, across the 0/2pi seam, on the rim,
near the origin and at R close to the filter's limit, that no decided pair
contradicts the oracle's FP64 predicate.  The same is done for the angular
windows in key units: every edge partner of a band lies inside the owner's
window, and every point inside its core is an edge, with the FP32 quotient,
rsqrt and asin taken at their documented error in the harmful direction.  The
constants are read from the CUDA sources, so the test follows them.
"""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1606_09481_gb300", "csrc")
f32, f64 = np.float32, np.float64


def _constants():
    src = open(os.path.join(CSRC, "common.cuh")).read() + open(os.path.join(CSRC, "query.cu")).read()
    out = {}
    for name in ("kEpsPM", "kEps32", "kCBase", "kAngAbs", "kC64", "kPiF", "kTwoPiHiF", "kTwoPiLoF"):
        m = re.search(r"constexpr float %s = ([-0-9.eE+]+)f;" % name, src)
        assert m, name
        out[name] = f32(float(m.group(1)))
    m = re.search(r"constexpr double kDeltaR = ([-0-9.eE+]+);", src)
    out["kDeltaR"] = float(m.group(1))
    m = re.search(r"constexpr int kExpTab = (\d+);", src)
    out["kExpTab"] = int(m.group(1))
    return out


C = _constants()


def fma(a, b, c):
    """fmaf: the float32 product is exact in float64, one rounding of the sum (a
    second rounding to float32 differs from a single one only at exact ties)."""
    return (np.asarray(a, f64) * np.asarray(b, f64) + np.asarray(c, f64)).astype(f32)


def filter_values(ph, r, G):
    """Angle hi/lo and (P, M, S, gamma) of points with FP64 angle ph and radius r."""
    K = C["kExpTab"]
    etab = np.exp(np.arange(-K, K + 1, dtype=f64)).astype(f32)
    hi = ph.astype(f32)
    lo = (ph - hi.astype(f64)).astype(f32)

    def exp_split(x):
        kd = np.rint(x)
        f = (x - kd).astype(f32)
        return (etab[kd.astype(np.int64) + K] * np.exp(f)).astype(f32)

    P, M = exp_split(r - G), exp_split(-r - G)
    big = r >= 1.0
    with np.errstate(divide="ignore", invalid="ignore"):
        S_big = ((P - M) * f32(0.70710678118654752)).astype(f32)
        g_big = (C["kEpsPM"] * ((P + M) / (P - M)) + f32(2.0) * C["kEps32"]).astype(f32)
        S_small = (np.sinh(r) * math.exp(-G) * 1.4142135623730951).astype(f32)
        g_small = (C["kEpsPM"] * (np.cosh(r) / np.sinh(r)).astype(f32) + f32(2.0) * C["kEps32"]).astype(f32)
    S = np.where(big, S_big, np.where(r > 0, S_small, f32(0))).astype(f32)
    gam = np.where(big, g_big, np.where(r > 0, g_small, f32(0))).astype(f32)
    return hi, lo, P, M, S, gam


def filter_decide(v, w):
    """1 = edge, 0 = no edge, 2 = undecided, for owner values v and candidate w
    (tuples from filter_values)."""
    vhi, vlo, Pv, Mv, Sv, gv = v
    whi, wlo, Pw, Mw, Sw, gw = w
    S2v, PMv, cv = (f32(2.0) * Sv).astype(f32), (Pv + Mv).astype(f32), (C["kCBase"] + gv).astype(f32)
    dh = (vhi - whi).astype(f32)
    d_plain = np.abs((dh + (vlo - wlo).astype(f32)).astype(f32))
    vbig = dh > 0
    bh, bl = np.where(vbig, vhi, whi), np.where(vbig, vlo, wlo)
    sh, sl = np.where(vbig, whi, vhi), np.where(vbig, wlo, vlo)
    d_wrap = ((((C["kTwoPiHiF"] - bh).astype(f32) + sh).astype(f32)
               + ((C["kTwoPiLoF"] - bl).astype(f32) + sl).astype(f32)).astype(f32))
    d = np.where(np.abs(dh) > C["kPiF"], d_wrap, d_plain).astype(f32)
    x = (f32(0.5) * d).astype(f32)
    z = (x * x).astype(f32)
    zx = (z * x).astype(f32)
    t_small = fma(zx, f32(-0.166666672), x)
    t = fma(z, f32(-2.50521079e-08), f32(2.75573188e-06))
    t = fma(z, t, f32(-1.98412701e-04))
    t = fma(z, t, f32(8.33333377e-03))
    t = fma(z, t, f32(-1.66666672e-01))
    t = np.where(x < f32(0.0078125), t_small, fma(zx, t, x)).astype(f32)
    ss = (S2v * Sw).astype(f32)
    sst = (ss * t).astype(f32)
    X = fma(sst, t, fma(Pv, Mw, (Mv * Pw).astype(f32)))
    err = fma(X, (cv + gw).astype(f32),
              fma((C["kC64"] * PMv).astype(f32), (Pw + Mw).astype(f32), (sst * C["kAngAbs"]).astype(f32)))
    return np.where((X + err).astype(f32) <= 1, 1, np.where((X - err).astype(f32) > 1, 0, 2))


def _pairs(rng, R, count):
    """Radii from several regimes, angles at the exact threshold angle times
    (1 + delta) with |delta| from 1e-9 to 1e-1, half of them across the seam."""
    kind = rng.integers(0, 4, count)
    rv = np.where(kind == 0, rng.uniform(0, R, count), np.where(kind == 1, R - rng.exponential(1.0, count),
                  np.where(kind == 2, rng.uniform(0, 1.5, count), R - rng.exponential(0.2, count))))
    rw = np.where(kind == 3, R - rng.exponential(0.2, count), R - rng.exponential(2.0, count))
    rv, rw = np.clip(rv, 0, R), np.clip(rw, 0, R)
    with np.errstate(divide="ignore", invalid="ignore"):
        A = (np.cosh(rv) * np.cosh(rw) - math.cosh(R)) / (np.sinh(rv) * np.sinh(rw))
    theta = np.arccos(np.clip(np.nan_to_num(A, nan=1.0), -1.0, 1.0))
    delta = rng.choice([-1.0, 1.0], count) * 10.0 ** rng.uniform(-9, -1, count)
    dphi = np.clip(theta * (1 + delta), 0, math.pi)
    phv = np.where(rng.random(count) < 0.5, rng.uniform(0, 1e-3, count), rng.uniform(0, 2 * math.pi, count))
    phw = np.mod(phv - dphi, 2 * math.pi)
    phw = np.where(phw >= 2 * math.pi, np.nextafter(2 * math.pi, 0), phw)
    return phv, rv, phw, rw, delta


@pytest.mark.parametrize("R", [0.7, 2.0, 3.0046, 16.705, 23.5089, 25.564, 31.9])
def test_filter_decisions_are_sound(O, R):
    rng = np.random.default_rng(int(R * 1000))
    n = 20000
    phv, rv, phw, rw, delta = _pairs(rng, R, n)
    G = 0.5 * math.log(2 * math.cosh(R))
    # the sampler's FP32-assisted radius is within kDeltaR / 2 of the FP64 one
    eps = C["kDeltaR"] * 0.54
    rva = np.clip(rv + rng.choice([-eps, eps, 0.0], n), 0, R)
    rwa = np.clip(rw + rng.choice([-eps, eps, 0.0], n), 0, R)
    dec = filter_decide(filter_values(phv, rva, G), filter_values(phw, rwa, G))
    truth = np.array([O.edge(phv[i], rv[i], phw[i], rw[i], R) for i in range(n)], dtype=np.int64)
    decided = dec != 2
    wrong = np.flatnonzero(decided & (dec != truth))
    assert wrong.size == 0, [(phv[i], rv[i], phw[i], rw[i], dec[i], truth[i]) for i in wrong[:5]]
    # and it is useful: far from the threshold most pairs are decided
    far = np.abs(delta) > 1e-2
    assert decided[far].mean() > 0.5
    assert truth.min() == 0 and truth.max() == 1


def test_emulation_flags_a_planted_error(O):
    """With the error bound removed (err = 0) the same pairs do contradict the
    FP64 predicate, so the sound result above is not vacuous."""
    R = 23.5089
    rng = np.random.default_rng(5)
    n = 20000
    phv, rv, phw, rw, delta = _pairs(rng, R, n)
    G = 0.5 * math.log(2 * math.cosh(R))
    saved = dict(C)
    try:
        C["kCBase"], C["kC64"], C["kAngAbs"], C["kEpsPM"], C["kEps32"] = (f32(0),) * 5
        dec = filter_decide(filter_values(phv, rv, G), filter_values(phw, rw, G))
    finally:
        C.update(saved)
    truth = np.array([O.edge(phv[i], rv[i], phw[i], rw[i], R) for i in range(n)], dtype=np.int64)
    assert np.count_nonzero((dec != 2) & (dec != truth)) > 0


# ---------------------------------------------------------------------------
# Windows in angle-key units (Sec. III-B getMinMaxPhi with the filter's error
# terms): every edge partner in band i lies within the window, and every point
# within the core is an edge.  The FP32 transcendentals (quotient, rsqrt, asin)
# are taken at their documented error, rounded in the direction that hurts.

def _cq():
    src = open(os.path.join(CSRC, "query.cu")).read() + open(os.path.join(CSRC, "common.cuh")).read()
    out = {}
    for name in ("kWinE1", "kNearMargin", "kKeyPerRadF"):
        m = re.search(r"constexpr float %s = ([-0-9.eE+]+)f;" % name, src)
        assert m, name
        out[name] = f32(float(m.group(1)))
    m = re.search(r"constexpr double kKeyScale = (0x[0-9a-fp+.-]+);", src)
    out["kKeyScale"] = float.fromhex(m.group(1))
    return out


W = _cq()
KFULL = 0x80000000


def bump(x, ulps):
    """x moved by |ulps| float32 ulps towards +inf (ulps > 0) or -inf."""
    x = np.asarray(x, f32)
    for _ in range(abs(ulps)):
        x = np.nextafter(x, f32(np.inf) if ulps > 0 else f32(-np.inf)).astype(f32)
    return x


def half_angle(Q, s):
    """asin(sqrt(Q)); s = -1 takes every approximate step at its low end, +1 high."""
    with np.errstate(divide="ignore", invalid="ignore"):
        rs = bump((1.0 / np.sqrt(np.asarray(Q, f64))).astype(f32), 2 * s)
        y = (Q * rs).astype(f32)
    y2 = (y * y).astype(f32)
    small = (y * fma(y2, fma(y2, f32(0.075), f32(0.16666667)), f32(1.0))).astype(f32)
    big = bump(np.arcsin(np.minimum(y, f32(1.0))).astype(f32), 2 * s)
    return np.where(Q > 0, np.where(y < f32(0.125), small, big), f32(0)).astype(f32)


def band_constants(R, c, i, G):
    sq = math.exp(-G)
    ci = max(c[i] - C["kDeltaR"], 0.0)
    co = c[i + 1] + C["kDeltaR"]
    return dict(P=f32(math.exp(ci) * sq), Mm=f32(math.exp(-ci) * sq), S=f32(math.sinh(ci) * sq * 1.4142135623730951),
                PMn=f32(2.0 * math.cosh(co) * sq * (1.0 + 1e-6)), Po=f32(math.exp(co) * sq),
                Mo=f32(math.exp(-co) * sq), So=f32(math.sinh(co) * sq * 1.4142135623730951))


def window_filter(v, B, i):
    _, _, P, M, S, gam = v
    S2, PM = (f32(2) * S).astype(f32), (P + M).astype(f32)
    T = fma(P, B["Mm"], (M * B["P"]).astype(f32))
    beta = fma((C["kC64"] * PM).astype(f32), B["PMn"], f32(1.0))
    num = fma((f32(1.0) + T).astype(f32), W["kWinE1"], (beta - T).astype(f32))
    den = ((S2 * B["S"]).astype(f32) * (f32(1.0) - (gam + f32(6.0) * C["kEps32"]).astype(f32))).astype(f32)
    with np.errstate(divide="ignore", invalid="ignore"):
        Q = bump((num / den).astype(f32), -2)
    full = (i == 0) | ~(B["S"] > 0) | ~(S2 > 0) | ~(Q < 1)
    th = half_angle(np.maximum(Q, f32(0)), -1)
    K = (W["kKeyPerRadF"] * (f32(2.0) * (f32(1.0) + f32(2e-5))).astype(f32)).astype(f32)
    keys = fma(th, K, f32(3.0))
    full |= keys >= f32(2147483648.0)
    return np.where(full, KFULL, np.floor(np.where(full, 0, keys)).astype(np.int64))


def window_core(v, B):
    _, _, P, M, S, gam = v
    S2, PM = (f32(2) * S).astype(f32), (P + M).astype(f32)
    m = fma((C["kC64"] * PM).astype(f32), B["PMn"], W["kNearMargin"])
    S2d = (S2 * (f32(1.0) + (gam + f32(6.0) * C["kEps32"]).astype(f32))).astype(f32)
    Q = np.full(P.shape, f32(4.0))
    none = np.zeros(P.shape, bool)
    for Pb, Mb, Sb in ((B["Po"], B["Mo"], B["So"]), (B["P"], B["Mm"], B["S"])):
        T = fma(P, Mb, (M * Pb).astype(f32))
        num = (((f32(1.0) - m).astype(f32) - T).astype(f32) - ((f32(1.0) + T).astype(f32) * W["kWinE1"]).astype(f32))
        none |= ~(num > 0)
        den = (S2d * Sb).astype(f32)
        with np.errstate(divide="ignore", invalid="ignore"):
            q = bump((num / den).astype(f32), 2)
        Q = np.where(den > 0, np.minimum(Q, q), Q).astype(f32)
    th = half_angle(Q, 1)
    K = (W["kKeyPerRadF"] * (f32(2.0) * (f32(1.0) - f32(4e-5))).astype(f32)).astype(f32)
    keys = ((th * K).astype(f32) - f32(4.0)).astype(f32)
    core = np.where(keys < 0, -1, np.floor(np.maximum(keys, 0)).astype(np.int64))
    core = np.where(Q >= 1, KFULL, core)
    return np.where(none, -1, core)


def angle_key(ph):
    t = np.floor(ph * W["kKeyScale"])
    return np.clip(t, 0, 4294967295).astype(np.int64)


@pytest.mark.parametrize("n,k,alpha", [(10_000, 6, 1.0), (10**7, 200, 1.0), (10**6, 16, 0.75), (5000, 60, 1.5)])
def test_windows_contain_every_edge_and_cores_only_edges(O, n, k, alpha):
    R = O.target_radius(n, k, alpha)
    B = O.default_bands(n)
    c = O.boundaries(R, B)
    G = 0.5 * math.log(2 * math.cosh(R))
    rng = np.random.default_rng(n + k)
    count = 20000
    eps = C["kDeltaR"] * 0.54
    checked = cores = 0
    for _ in range(4):
        i = rng.integers(1, B, count)  # candidate band (band 0 is always searched whole)
        # the sampler's radius of w: in band i, a third at each edge of the band
        u = rng.random(count)
        u = np.where(rng.random(count) < 0.33, 0.0, np.where(rng.random(count) < 0.5, 1.0 - 1e-12, u))
        rw_a = c[i] + (c[i + 1] - c[i]) * u
        rw = np.clip(rw_a + rng.uniform(-eps, eps, count), 0, R)
        bv = (rng.random(count) * (i + 1)).astype(np.int64)  # v in band i or inside it
        rv_a = np.minimum(c[bv] + (c[bv + 1] - c[bv]) * rng.random(count), R)
        rv = np.clip(rv_a + rng.uniform(-eps, eps, count), 0, R)
        with np.errstate(divide="ignore", invalid="ignore"):
            A = (np.cosh(rv) * np.cosh(rw) - math.cosh(R)) / (np.sinh(rv) * np.sinh(rw))
        theta = np.arccos(np.clip(np.nan_to_num(A, nan=1.0), -1.0, 1.0))
        # a quarter of the pairs anywhere inside the threshold angle, the rest at it
        near = theta * (1 + rng.choice([-1, 1], count) * 10.0 ** rng.uniform(-9, -0.5, count))
        dphi = np.clip(np.where(rng.random(count) < 0.25, theta * rng.random(count), near), 0, math.pi)
        S = 2 * math.pi * 2.0 ** -53
        uv = rng.integers(0, 2**53, count, dtype=np.int64)
        uw = np.mod(uv + np.rint(rng.choice([-1, 1], count) * dphi / S).astype(np.int64), 2**53)
        phv, phw = uv.astype(f64) * S, uw.astype(f64) * S
        # keys of loaded points (floor of phi 2^32 / 2pi) and of generated points
        # (the top 32 bits of the 53-bit angle draw): the window must hold the
        # larger distance, the core must exclude non-edges at the smaller one
        dists = []
        for kv, kw in ((angle_key(phv), angle_key(phw)), (uv >> 21, uw >> 21)):
            d = np.abs(kv - kw)
            dists.append(np.minimum(d, 2**32 - d))
        kd, kd_core = np.maximum(*dists), np.minimum(*dists)
        v = filter_values(phv, rv_a, G)
        for band in np.unique(i):
            sel = np.flatnonzero(i == band)
            Bc = band_constants(R, c, band, G)
            vs = tuple(a[sel] for a in v)
            wf = window_filter(vs, Bc, band)
            wc = window_core(vs, Bc)
            truth = np.array([O.edge(phv[j], rv[j], phw[j], rw[j], R) for j in sel], dtype=bool)
            inside = (wf == KFULL) | (kd[sel] <= wf)
            missed = sel[truth & ~inside]
            assert missed.size == 0, [(rv[j], rw[j], kd[j], band) for j in missed[:5]]
            plain = wf < KFULL
            core = np.where(wc == KFULL, wf, np.minimum(wc, wf))
            in_core = plain & (wc >= 0) & (kd_core[sel] <= core)
            bad = sel[in_core & ~truth]
            assert bad.size == 0, [(rv[j], rw[j], kd[j], band) for j in bad[:5]]
            checked += sel.size
            cores += int(in_core.sum())
    assert cores > 0.05 * checked  # the core test is not vacuous


def test_window_checks_detect_planted_errors(O, monkeypatch):
    """A window 10^-4 too narrow, or a core 10^-4 too wide, fails the check
    above: its pairs come close enough to the band edges and the threshold."""
    import sys
    mod = sys.modules[__name__]
    wf0, wc0 = mod.window_filter, mod.window_core

    def narrow(v, B, i):
        w = wf0(v, B, i)
        return np.where(w < KFULL, np.floor(w * (1 - 1e-4) - 8).astype(np.int64), w)

    def wide(v, B):
        w = wc0(v, B)
        return np.where((w >= 0) & (w < KFULL), np.floor(w * (1 + 1e-4) + 8).astype(np.int64), w)

    for name, fake in (("window_filter", narrow), ("window_core", wide)):
        with monkeypatch.context() as m:
            m.setattr(mod, name, fake)
            with pytest.raises(AssertionError):
                test_windows_contain_every_edge_and_cores_only_edges(O, 10**7, 200, 1.0)


# ---------------------------------------------------------------------------
# The sampler's FP32-assisted radius (band assignment and filter values): within
# kDeltaR of the FP64 radius for every alpha > 1/2 and alpha R up to the filter's
# limit, with logf taken 2 ulp off in either direction.

def radius_approx(u53, R, alpha, s):
    cm1 = math.cosh(alpha * R) - 1.0
    U = u53.astype(f64) * 2.0 ** -53
    wf = (U * cm1).astype(f32)
    y = ((f32(1.0) + wf).astype(f32) + np.sqrt((wf * (wf + f32(2.0)).astype(f32)).astype(f32))).astype(f32)
    m, e = np.frexp(y)
    low = m < f32(0.70710678)
    m = np.where(low, (m * f32(2.0)).astype(f32), m).astype(f32)
    e = np.where(low, e - 1, e)
    lg = e.astype(f64) * 0.69314718055994530942 + bump(np.log(m).astype(f32), 2 * s).astype(f64)
    r = lg * (1.0 / alpha)
    return np.where(r < R, np.maximum(r, 0.0), R)


@pytest.mark.parametrize("alpha,R", [(0.51, 30.0), (0.55, 25.0), (0.75, 25.564), (1.0, 23.5089), (1.5, 16.0),
                                     (3.0, 14.66), (1.375, 32.0), (1.0, 31.9), (0.51, 3.0), (1.0, 2.0)])
def test_sampler_radius_within_kDeltaR(alpha, R):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    rng = np.random.default_rng(int(alpha * 100 + R))
    u53 = np.concatenate([rng.integers(0, 2**53, 3000, dtype=np.int64),
                          (2.0 ** rng.uniform(0, 53, 1000)).astype(np.int64),
                          np.array([0, 1, 2, 3, 2**20, 2**40, 2**52, 2**53 - 2, 2**53 - 1], dtype=np.int64)])
    cm1 = mpmath.cosh(mpmath.mpf(alpha) * R) - 1
    exact = np.array([float(mpmath.acosh(1 + mpmath.mpf(int(u)) / 2**53 * cm1) / alpha) for u in u53])
    exact = np.minimum(exact, R)
    for s in (-1, 0, 1):
        err = np.abs(radius_approx(u53, R, alpha, s) - exact)
        assert err.max() <= 5.4e-7, (s, err.max(), u53[err.argmax()])
    assert 5.4e-7 < C["kDeltaR"]


def test_filter_range_keeps_the_sampler_radius_finite():
    """The filter is used only for alpha R <= kFilterMaxAlphaR; there the FP32
    w (w + 2) of the approximate radius must not overflow (it would put every
    point at R), and just above the limit it would."""
    src = open(os.path.join(CSRC, "common.cuh")).read()
    lim = float(re.search(r"constexpr double kFilterMaxAlphaR = ([0-9.]+);", src).group(1))
    for aR, finite in ((lim, True), (45.2, False)):
        wf = f32(math.cosh(aR) - 1.0)
        with np.errstate(over="ignore"):
            prod = (wf * (wf + f32(2.0)).astype(f32)).astype(f32)
        assert np.isfinite(prod) == finite, aR
    # at the limit the approximate radius of the largest variate is still right
    alpha, R = 1.375, lim / 1.375
    r = radius_approx(np.array([2**53 - 1], dtype=np.int64), R, alpha, 0)
    assert abs(r[0] - R) < 5.4e-7


def window_fp64(rv, c, i, R):
    """The FP64-mode half-width in key units (kFull: the whole band)."""
    chv, shv = np.cosh(rv), np.sinh(rv)
    u = 2.0 ** -53
    b = (math.cosh(R) + 64.0 * u * chv * math.cosh(c[i + 1])) * (1.0 + 1e-12)
    with np.errstate(divide="ignore", invalid="ignore"):
        Q = (b - np.cosh(rv - c[i])) / (2.0 * shv * math.sinh(c[i]))
    full = (c[i] <= 0) | (rv <= 0) | (shv <= 0) | ~(Q < 1.0)
    with np.errstate(invalid="ignore"):
        th = 2.0 * np.arcsin(np.sqrt(np.where(Q > 0, Q, 0.0))) * (1.0 + 1e-9) + 1e-12
    keys = th * 683565275.57643158 + 3.0
    full |= keys >= 2147483648.0
    return np.where(full, KFULL, np.floor(np.where(full, 0, keys)).astype(np.int64))


@pytest.mark.parametrize("n,k,alpha", [(5000, 2, 3.0), (3000, 2, 5.0), (10**6, 1, 0.6), (10**4, 6, 1.0)])
def test_fp64_windows_contain_every_edge(O, n, k, alpha):
    """FP64 mode (bands from the FP64 radius): every edge partner in band i lies
    within the owner's window, at both edges of the band and at the threshold."""
    R = O.target_radius(n, k, alpha)
    B = O.default_bands(n)
    c = O.boundaries(R, B)
    rng = np.random.default_rng(n + 7)
    count = 40000
    i = rng.integers(1, B, count)
    u = rng.random(count)
    u = np.where(rng.random(count) < 0.33, 0.0, np.where(rng.random(count) < 0.5, 1.0 - 1e-12, u))
    rw = c[i] + (c[i + 1] - c[i]) * u
    bv = (rng.random(count) * (i + 1)).astype(np.int64)
    rv = np.minimum(c[bv] + (c[bv + 1] - c[bv]) * rng.random(count), R)
    with np.errstate(divide="ignore", invalid="ignore"):
        A = (np.cosh(rv) * np.cosh(rw) - math.cosh(R)) / (np.sinh(rv) * np.sinh(rw))
    theta = np.arccos(np.clip(np.nan_to_num(A, nan=1.0), -1.0, 1.0))
    dphi = np.clip(theta * (1 - 10.0 ** rng.uniform(-12, -1, count)), 0, math.pi)
    S = 2 * math.pi * 2.0 ** -53
    uv = rng.integers(0, 2**53, count, dtype=np.int64)
    uw = np.mod(uv + np.rint(rng.choice([-1, 1], count) * dphi / S).astype(np.int64), 2**53)
    phv, phw = uv.astype(f64) * S, uw.astype(f64) * S
    kd = np.zeros(count, np.int64)
    for kv, kw in ((angle_key(phv), angle_key(phw)), (uv >> 21, uw >> 21)):
        d = np.abs(kv - kw)
        kd = np.maximum(kd, np.minimum(d, 2**32 - d))
    truth = np.array([O.edge(phv[j], rv[j], phw[j], rw[j], R) for j in range(count)], dtype=bool)
    wf = np.empty(count, np.int64)
    for band in np.unique(i):
        sel = i == band
        wf[sel] = window_fp64(rv[sel], c, band, R)
    missed = np.flatnonzero(truth & ~((wf == KFULL) | (kd <= wf)))
    assert missed.size == 0, [(rv[j], rw[j], kd[j], wf[j]) for j in missed[:5]]
    assert truth.mean() > 0.5  # most pairs sit just inside the threshold


def test_fp64_window_check_detects_a_planted_error(O, monkeypatch):
    """The same check fails for a window only 4 keys narrower."""
    import sys
    mod = sys.modules[__name__]
    w0 = mod.window_fp64

    def narrow(rv, c, i, R):
        w = w0(rv, c, i, R)
        return np.where(w < KFULL, w - 4, w)

    monkeypatch.setattr(mod, "window_fp64", narrow)
    with pytest.raises(AssertionError):
        test_fp64_windows_contain_every_edge(O, 10**4, 6, 1.0)
