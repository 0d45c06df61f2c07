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


# Largest relative error of the stored P and M of a generated point
# (filter_values_u53: y from the variate in FP32, then the exponent tables),
# established by test_generated_filter_values_within_the_bound below; the
# decision and window checks perturb P and M by it.
EPS_PM_U53 = 1.2e-6


def filter_values(ph, r, G, eP=0.0, eM=0.0, er=0.0):
    """Angle hi/lo and (P, M, S, gamma) of points with FP64 angle ph and radius r;
    P and M multiplied by (1 + eP), (1 + eM) and the radius of the small-r
    branch shifted by er (the stored values' errors)."""
    K = C["kExpTab"]
    etab = np.exp(np.arange(-K, K + 1, dtype=f64)).astype(f32)
    hi = ph.astype(f32)
    lo = (ph - hi.astype(f64)).astype(f32)

    def exp_split(x):
        kd = np.rint(x)
        f = (x - kd).astype(f32)
        return (etab[kd.astype(np.int64) + K] * np.exp(f)).astype(f32)

    P = (exp_split(r - G) * (1.0 + np.asarray(eP, f64))).astype(f32)
    M = (exp_split(-r - G) * (1.0 + np.asarray(eM, f64))).astype(f32)
    r = np.clip(r + er, 0.0, None)
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
    # stored P and M within EPS_PM_U53 (relative) of the exact ones, the small-r
    # branch's radius within 6 u / alpha (alpha > 1/2)
    e, er = EPS_PM_U53, 12 * 2.0 ** -24

    def err():
        return rng.choice([-e, e, 0.0], n), rng.choice([-e, e, 0.0], n), rng.choice([-er, er, 0.0], n)

    dec = filter_decide(filter_values(phv, rv, G, *err()), filter_values(phw, rw, G, *err()))
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
        # the owner's stored values: P and M within EPS_PM_U53 of those of its radius
        # rv (a third low, a third high, a third exact)
        ev = rng.choice([-EPS_PM_U53, EPS_PM_U53, 0.0], (2, count))
        v = filter_values(phv, rv, G, ev[0], ev[1], rng.choice([-12, 12, 0], count) * 2.0 ** -24)
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
# Generated points in filter mode: the band from the radial variate and the
# filter values from the variates, without FP64 (band_of_u53, angle_hilo_u53,
# filter_values_u53), restated operation by operation.

K_SIG = 0x1921FB54442D18  # significand of 2 pi: kPhiScale = K_SIG 2^-103


def angle_hilo_u53(u):
    """The device's integer construction of the angle's hi/lo floats."""
    if u == 0:
        return 0.0, 0.0
    prod = u * K_SIG
    sh = prod.bit_length() - 53
    q, rem = prod >> sh, prod & ((1 << sh) - 1)
    if sh and (rem > (1 << (sh - 1)) or (rem == (1 << (sh - 1)) and q & 1)):
        q += 1
        if q == 1 << 53:
            q >>= 1
            sh += 1
    if sh > 53 or (sh == 53 and q >= K_SIG):
        q, sh = K_SIG - 1, 53
    h, r = q >> 29, q & ((1 << 29) - 1)
    if r > (1 << 28) or (r == (1 << 28) and h & 1):
        h += 1
    lo_i = q - (h << 29)
    hi = float(np.float32(h)) * 2.0 ** (sh - 74)
    lo = float(np.float32(lo_i)) * 2.0 ** (sh - 103)  # int -> float rounds to nearest even
    return hi, lo


def test_generated_angle_pair_is_the_fp64_pair():
    """The integer construction gives bit for bit the pair float(phi),
    float(phi - float(phi)) of phi = fl(u53 * 2pi 2^-53) (clamped below 2 pi):
    small variates (many rounding ties), random ones, and the extremes."""
    rng = np.random.default_rng(53)
    us = np.concatenate([np.arange(0, 4096), rng.integers(0, 2**53, 60000, dtype=np.int64),
                         (2.0 ** rng.uniform(0, 53, 20000)).astype(np.int64),
                         np.array([2**52, 2**52 + 1, 2**53 - 2, 2**53 - 1, 2**29 + 2**28], dtype=np.int64)])
    two_pi = float.fromhex("0x1.921fb54442d18p+2")
    ph = us.astype(f64) * float.fromhex("0x1.921fb54442d18p-51")
    ph = np.where(ph < two_pi, ph, np.nextafter(two_pi, 0.0))
    hi = ph.astype(f32)
    lo = (ph - hi.astype(f64)).astype(f32)
    got = np.array([angle_hilo_u53(int(u)) for u in us])
    assert np.array_equal(got[:, 0].astype(f32), hi) and np.array_equal(got[:, 1].astype(f32), lo)
    # the restatement is exact in float64 (powers of two times <= 29-bit integers)
    assert np.array_equal(got[:, 0], hi.astype(f64)) and np.array_equal(got[:, 1], lo.astype(f64))


def _cm1(O, alpha, R):
    return float(O.dm("cosh", np.array([alpha * R]))[0]) - 1.0


def filter_values_u53(O, ur, alpha, R, s_log=0, s_exp=0):
    """P, M, S, gamma of generated points from their radial variates, as the
    device computes them; log2f and exp2f moved by their documented largest
    errors (1 and 2 ulp) in the direction s_log, s_exp."""
    G = 0.5 * math.log(2.0 * float(O.dm("cosh", np.array([R]))[0]))
    cm1 = _cm1(O, alpha, R)
    cw = f32(cm1 * 2.0 ** -53)
    uf = ur.astype(f64).astype(f32)  # exact in float64, one rounding to float32
    wf = (uf * cw).astype(f32)
    y = ((f32(1) + wf).astype(f32) + np.sqrt((wf * (wf + f32(2)).astype(f32)).astype(f32))).astype(f32)
    m, e = np.frexp(y)
    low = m < f32(0.70710678)
    m = np.where(low, (m * f32(2)).astype(f32), m).astype(f32)
    e = np.clip(np.where(low, e - 1, e), 0, 65)
    ea = e * 0.69314718055994530942 / alpha
    tabP = np.minimum(np.exp(ea - G), 3.0e38).astype(f32)
    tabM = np.exp(-ea - G).astype(f32)
    if alpha == 1.0:
        mp, mm = m, (f32(1) / m).astype(f32)
    else:
        ia = f32(1.0 / alpha)
        t = (bump(np.log2(m).astype(f32), s_log) * ia).astype(f32)
        mp = bump(np.exp2(t).astype(f32), 2 * s_exp)
        mm = bump(np.exp2(-t).astype(f32), 2 * s_exp)
    P = (tabP * mp).astype(f32)
    M = (tabM * mm).astype(f32)
    y_one = f32(math.exp(alpha))
    with np.errstate(divide="ignore", invalid="ignore"):
        S_big = ((P - M) * f32(0.70710678118654752)).astype(f32)
        g_big = (C["kEpsPM"] * ((P + M) / (P - M)) + f32(2) * C["kEps32"]).astype(f32)
        r = np.log(y.astype(f64)) * (1.0 / alpha)
        S_small = (np.sinh(r) * math.exp(-G) * 1.4142135623730951).astype(f32)
        g_small = (C["kEpsPM"] * (np.cosh(r) / np.sinh(r)).astype(f32) + f32(2) * C["kEps32"]).astype(f32)
    S = np.where(y >= y_one, S_big, np.where(y > f32(1), S_small, f32(0))).astype(f32)
    gam = np.where(y >= y_one, g_big, np.where(y > f32(1), g_small, f32(0))).astype(f32)
    return P, M, S, gam, y, G


def _variates(rng):
    return np.concatenate([rng.integers(0, 2**53, 1500, dtype=np.int64),
                           (2.0 ** rng.uniform(0, 53, 700)).astype(np.int64),
                           np.array([0, 1, 2, 3, 2**20, 2**40, 2**52, 2**53 - 2, 2**53 - 1], dtype=np.int64)])


@pytest.mark.parametrize("alpha,R", [(0.51, 30.0), (0.55, 25.0), (0.75, 25.564), (1.0, 23.5089), (1.5, 16.0),
                                     (3.0, 14.66), (1.375, 32.0), (1.0, 31.9), (0.51, 3.0), (1.0, 2.0)])
def test_generated_filter_values_within_the_bound(O, alpha, R):
    """P = e^{r - G} and M = e^{-r - G} of generated points, formed from y in FP32
    and the exponent tables, stay within EPS_PM_U53 < kEpsPM of the exact values
    of the point's radius (inverse CDF of Eq. 1 in 120-bit arithmetic), and S
    within its stored bound gamma, for every alpha > 1/2 and alpha R up to the
    filter's limit, with log2f / exp2f at either end of their error."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    assert EPS_PM_U53 < float(C["kEpsPM"])
    rng = np.random.default_rng(int(alpha * 100 + R))
    ur = _variates(rng)
    cm1 = mpmath.mpf(_cm1(O, alpha, R))
    Gm = None
    exact = []
    for u in ur:
        r = mpmath.acosh(1 + mpmath.mpf(int(u)) / 2**53 * cm1) / alpha
        exact.append(min(r, mpmath.mpf(R)))
    worst = 0.0
    for s_log in (-1, 0, 1):
        for s_exp in (-1, 0, 1):
            P, M, S, gam, y, G = filter_values_u53(O, ur, alpha, R, s_log, s_exp)
            if Gm is None:
                Gm = mpmath.mpf(G)
                Pe = np.array([float(mpmath.exp(r - Gm)) for r in exact])
                Me = np.array([float(mpmath.exp(-r - Gm)) for r in exact])
                Se = np.array([float(mpmath.sinh(r) * mpmath.exp(-Gm) * mpmath.sqrt(2)) for r in exact])
            eP = np.abs(P.astype(f64) / Pe - 1)
            eM = np.abs(M.astype(f64) / Me - 1)
            worst = max(worst, eP.max(), eM.max())
            assert eP.max() <= EPS_PM_U53 and eM.max() <= EPS_PM_U53, (s_log, s_exp, eP.max(), eM.max())
            # S within gamma (relative) where y > 1; where y rounds to 1 the point is
            # stored at r = 0 (S = 0, gamma = 0) and its true radius is below
            # 12 u / alpha: an absolute error of S that the relative term of the
            # filter's bound covers (X >= (P_v + M_v) e^{-G} ~ 2 S_v e^{-G}/sqrt 2)
            pos = y > f32(1)
            eS = np.abs(S.astype(f64)[pos] / Se[pos] - 1)
            assert np.all(eS <= gam.astype(f64)[pos]), (s_log, s_exp, (eS - gam[pos]).max())
            r0 = np.array([float(r) for r in exact])[~pos]
            assert np.all(S[~pos] == 0) and np.all(r0 <= 12 * 2.0 ** -24 / alpha)
    assert worst > 0.02 * EPS_PM_U53  # the comparison is not vacuous


def test_generated_filter_values_bound_is_tight_enough_to_catch_a_dropped_term(O):
    """A planted mistake in the restatement (the table without the e^-G factor's
    rounding direction, here y used without its sqrt term) breaks the bound."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    alpha, R = 1.0, 23.5089
    ur = _variates(np.random.default_rng(7))
    P, M, S, gam, y, G = filter_values_u53(O, ur, alpha, R)
    cm1 = mpmath.mpf(_cm1(O, alpha, R))
    # y without the sqrt term: 1 + w, about half of y for large w
    wf = (ur.astype(f64).astype(f32) * f32(float(cm1) * 2.0 ** -53)).astype(f32)
    bad_y = (f32(1) + wf).astype(f32)
    bad_P = (bad_y.astype(f64) * math.exp(-G))
    Pe = np.array([float(mpmath.exp(mpmath.acosh(1 + mpmath.mpf(int(u)) / 2**53 * cm1) / alpha - mpmath.mpf(G)))
                   for u in ur])
    assert np.abs(bad_P / Pe - 1).max() > EPS_PM_U53
    assert np.abs(P.astype(f64) / Pe - 1).max() <= EPS_PM_U53


def band_thresholds(c, alpha, cm1):
    """The plan's band thresholds on the radial variate: ceil(F(c_j) 2^53)."""
    B = len(c) - 1
    bu = np.zeros(B + 1, dtype=np.int64)
    for j in range(1, B):
        sh = math.sinh(0.5 * alpha * c[j])
        T = math.ceil(2.0 * sh * sh / cm1 * 2.0 ** 53)
        bu[j] = min(max(T, 0), 2**53)
    bu[B] = 2**53
    return bu


@pytest.mark.parametrize("n,k,alpha", [(10**7, 200, 1.0), (10**6, 16, 0.75), (5000, 60, 1.5), (10**5, 8, 0.55)])
def test_band_thresholds_bound_the_radius(O, n, k, alpha):
    """A variate at or above the threshold of band j has radius >= c_j - 1e-13, one
    below the threshold of band j + 1 has radius <= c_{j+1} + 1e-13 (radius: the
    oracle's FP64 inverse CDF), checked at every threshold and on random variates;
    a threshold one step too low (planted) puts a radius below its band."""
    R = O.target_radius(n, k, alpha)
    B = O.default_bands(n)
    c = O.boundaries(R, B)
    cm1 = _cm1(O, alpha, R)
    bu = band_thresholds(c, alpha, cm1)
    assert np.all(np.diff(bu) >= 0)
    rng = np.random.default_rng(n % 1000 + k)
    near = np.concatenate([bu[1:B, None] + np.arange(-3, 4)[None, :]]).ravel()
    us = np.concatenate([near, rng.integers(0, 2**53, 5000, dtype=np.int64),
                         (2.0 ** rng.uniform(0, 53, 2000)).astype(np.int64)])
    us = np.clip(us, 0, 2**53 - 1)
    r = O.radius_from_u53(us, alpha, R)
    band = np.searchsorted(bu, us, side="right") - 1
    assert np.all(band >= 0) and np.all(band < B)
    assert np.all(r >= c[band] - 1e-13) and np.all(r <= c[band + 1] + 1e-13)
    # the thresholds are tight: one below band j's threshold lies below c_j
    below = O.radius_from_u53(np.maximum(bu[1:B] - 1, 0), alpha, R)
    assert np.all(below <= c[1:B] + 1e-13)
    low = bu.copy()
    low[1:B] = np.maximum(low[1:B] - max(1, int(2**53 * 1e-9)), 0)
    band = np.searchsorted(low, us, side="right") - 1
    assert np.any(r < c[band] - 1e-13)


def test_filter_range_keeps_y_finite():
    """The filter is used only for alpha R <= kFilterMaxAlphaR; there the FP32
    w (w + 2) of y must not overflow (it would make every y infinite), and just
    above the limit it would."""
    src = open(os.path.join(CSRC, "common.cuh")).read()
    lim = float(re.search(r"constexpr double kFilterMaxAlphaR = ([0-9.]+);", src).group(1))
    for aR, finite in ((lim, True), (45.2, False)):
        wf = f32(math.cosh(aR) - 1.0)
        with np.errstate(over="ignore"):
            prod = (wf * (wf + f32(2.0)).astype(f32)).astype(f32)
        assert np.isfinite(prod) == finite, aR
    # and y's exponent stays inside the tables: y < 2^65
    y = f32(2) * f32(math.cosh(lim)) + f32(2)
    assert np.frexp(y)[1] <= 65


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
