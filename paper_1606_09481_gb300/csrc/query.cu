// query.cu -- the range query of Alg. 1, the loop that dominates the running time
// (Sec. III-B): for each point v and each band b_i from v's own band outward, the
// getMinMaxPhi window, a binary search for the first and last candidate in the
// band's angle-sorted keys, and the distance test of every candidate (Eq. 3).
//
// Work decomposition (GB300): a warp takes a batch of 32 consecutive sorted points
// (lane = point) and walks the bands.  For each band every lane computes
//  - the window of Sec. III-B from the band's inner radius (every neighbour is
//    inside), and
//  - a core window from both band radii: X = cosh(r_v - r_w)/cosh R + 2 sinh r_v
//    sinh r_w sin^2(d/2)/cosh R is convex in r_w, so it is largest at a band
//    radius, and a pair whose angle is inside the core is an edge for every r_w
//    of the band, including the rounding of the FP64 predicate;
// and queues the core range (certain edges, written without a test) and the
// fringe ranges (window minus core, tested).  A flush streams the core ranges to
// the output and lets all 32 lanes test the fringe candidates as one flat
// stream, one decision bit per candidate, reserves the output with one atomic
// add per segment and replays the bits to write the pairs.  Long ranges go to a
// chunk list that a second kernel spreads over all warps (hub vertices).
//
// Candidate test: in filter mode an FP32 test of X = L / cosh R written without
// cancellation, X = P_v M_w + M_v P_w + 2 S_v S_w sin^2(d/2), that decides only when
// |X - 1| exceeds a bound on all errors, including the rounding of the FP64
// predicate itself; undecided pairs are queued and the third kernel evaluates the
// FP64 predicate on them.  FP64 mode tests every candidate with the FP64 predicate.
#include "kernels.h"
#include "stages.cuh"

namespace rhg {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kChunk = 4096;      // candidates per heavy chunk
constexpr int kListCap = 64;           // queued fringe entries per warp (>= 2 per lane)
constexpr int kBitWords = 128;         // decision words per warp: kChunk / 32
constexpr uint32_t kFull = 0x80000000u;  // window half-width meaning "whole band"
constexpr int kBatchMinBlocks = 4;         // resident CTAs per SM the batch kernel is compiled for
constexpr int kCoreUnroll = 4;             // core-writer steps whose id loads are issued together
constexpr int kHeavyGroup = 16;            // the same in the heavy kernel's core chunks
constexpr int kFringeRounds = 4;           // heavy fringe-chunk rounds whose values load together

constexpr float kPiF = 3.14159265f;             // 3.14159274f, just above pi; sin^2(d/2) is even about pi
constexpr float kTwoPiHiF = 6.28318548202514648f;
constexpr float kTwoPiLoF = -1.74845553e-07f;    // 2 pi - kTwoPiHiF
constexpr float kKeyPerRadF = 683565248.0f;      // 2^32 / (2 pi) in FP32 (slightly low)
constexpr double kKeyPerRad = 683565275.57643158;
constexpr float kWinE1 = 5e-6f;                  // window numerator error, relative to 1 + T
constexpr float kNearMargin = 2e-12f;            // core pairs stay clear of |L/cosh R - 1| <= 1e-12

// Diagnostics of a pair decided by the FP64 predicate (reported, never used to
// decide): bit 0.. counts |L - cosh R| <= 1e-12 cosh R, bit 32.. counts
// |L - cosh R| <= 8 u cosh r_v cosh r_w (the predicate's rounding band).  Every
// pair inside the rounding band reaches the FP64 predicate: the filter and the
// core decide only pairs farther than 32 u cosh r_v cosh r_w from the threshold.
__device__ __forceinline__ uint64_t diag_count(double L, double coshR, double chv, double chw)
{
    const double dev = fabs(__dsub_rn(L, coshR));
    return (dev <= 1e-12 * coshR ? 1ull : 0ull) + (dev <= 0x1p-50 * __dmul_rn(chv, chw) ? (1ull << 32) : 0ull);
}

// Adds a warp's diagnostic counts (lane sums in `near`) to the graph's counters.
__device__ __forceinline__ void flush_diag(Meta *C, uint64_t near)
{
    for (int off = 16; off; off >>= 1) near += __shfl_down_sync(0xffffffffu, near, off);
    if ((threadIdx.x & 31) == 0 && near) {
        if (near & 0xffffffffull)
            atomicAdd(reinterpret_cast<unsigned long long *>(&C->near_threshold), near & 0xffffffffull);
        if (near >> 32) atomicAdd(reinterpret_cast<unsigned long long *>(&C->rounding_band), near >> 32);
    }
}

struct BandShared {
    uint32_t start[kMaxBands + 1];
    float P[kMaxBands + 1], Mm[kMaxBands + 1], S[kMaxBands + 1];     // inner radius c_i - dr
    float Po[kMaxBands + 1], Mo[kMaxBands + 1], So[kMaxBands + 1];   // outer radius c_{i+1} + dr
    float PMn[kMaxBands + 1];
    double c[kMaxBands + 1], sinh_c[kMaxBands + 1], cosh_c[kMaxBands + 1];
    uint32_t ioff[kMaxBands + 1], ishift[kMaxBands + 1];  // bucket index of each band
    uint32_t budget, core_heavy, fringe_limit;              // work mapping (Meta)
};

__device__ __forceinline__ void load_bands_from(BandShared &S, const Meta *M, int first, int stride)
{
    for (int j = first; j <= kMaxBands; j += stride) {
        S.start[j] = static_cast<uint32_t>(M->band_start[j]);
        S.P[j] = M->band_P[j];
        S.Mm[j] = M->band_M[j];
        S.S[j] = M->band_S[j];
        S.Po[j] = M->band_Po[j];
        S.Mo[j] = M->band_Mo[j];
        S.So[j] = M->band_So[j];
        S.PMn[j] = M->band_PMn[j];
        S.c[j] = M->c[j];
        S.sinh_c[j] = M->sinh_c[j];
        S.cosh_c[j] = M->cosh_c[j];
        S.ioff[j] = M->idx_off[j];
        S.ishift[j] = j < kMaxBands ? M->idx_shift[j] : 32u;
    }
    if (first == 0) {
        S.budget = M->batch_budget;
        S.core_heavy = M->core_heavy;
        S.fringe_limit = M->fringe_limit;
    }
}

__device__ __forceinline__ void load_bands(BandShared &S, const Meta *M) { load_bands_from(S, M, threadIdx.x, blockDim.x); }

// The values of a range's owner (the point whose neighbours are searched) that
// its lane keeps in registers for the windows.
struct OwnerRegs {
    float P, M, S2, PM, gam;  // filter mode
    double r, ch, sh;         // FP64 mode
};

// Per-warp shared state.  Queued fringe entries form a flat candidate stream:
// entry e holds stream positions pre[e] .. pre[e+1]-1 at sorted positions
// lo[e] + (j - pre[e]).  Owners by lane.
struct WarpSmem {
    uint32_t lo[kListCap], pre[kListCap + 1];
    uint8_t own[kListCap];
    float4 oa[32];      // filter owner: angle hi, angle lo, P, M
    float4 ob[32];      // filter owner: 2 S, P + M, kCBase + gamma, unused
    double2 od[32];     // FP64 owner: phi, cosh r
    double osh[32];     // FP64 owner: sinh r
    uint32_t opos[32];  // owner sorted position
    uint32_t oid[32];   // owner vertex id
    uint32_t bits[kBitWords];
    uint8_t round_entry[kBitWords];  // entry holding the first candidate of each round
};

// Load point p as the owner in slot `slot` (and return the window values).
template <bool kFilter>
__device__ __forceinline__ OwnerRegs load_owner(const SortedPoints &P, WarpSmem &W, int slot, uint32_t p)
{
    OwnerRegs o;
    W.opos[slot] = p;
    W.oid[slot] = P.id[p];
    if (kFilter) {
        const float2 a = P.ang[p];
        const float4 q = P.pms[p];
        o.P = q.x;
        o.M = q.y;
        o.S2 = 2.0f * q.z;
        o.PM = q.x + q.y;
        o.gam = q.w;
        W.oa[slot] = make_float4(a.x, a.y, q.x, q.y);
        W.ob[slot] = make_float4(o.S2, o.PM, kCBase + q.w, 0.0f);
    } else {
        o.r = P.r[p];
        o.ch = P.ch[p];
        o.sh = P.sh[p];
        W.od[slot] = make_double2(P.phi[p], o.ch);
        W.osh[slot] = o.sh;
    }
    return o;
}

// FP32 filter: 1 = edge, 0 = no edge, 2 = undecided (FP64 recheck).
//   d    circular |phi_v - phi_w| from hi/lo floats (relative error ~2^-23 plus an
//        absolute error < kAngAbs / 2 from the hi/lo representation)
//   t    sin(d/2): x - x^3/6 below x = 2^-7 (relative error < x^4/120 < 4e-11),
//        else the odd Taylor polynomial to x^11 on [0, pi/2] (~3 ulp)
//   X    P_v M_w + M_v P_w + 2 S_v S_w t^2
//   err  X (kCBase + gamma_v + gamma_w) + kC64 (P_v + M_v)(P_w + M_w)
//        + 2 S_v S_w t kAngAbs (the absolute angle error)
__device__ __forceinline__ int filter_decide(float4 va, float4 vb, float2 aw, float4 w)
{
    const float dh = va.x - aw.x;  // correctly rounded: relative error <= 2^-24
    float d;
    if (fabsf(dh) > kPiF) {
        // across 0 / 2 pi: 2 pi - (big - small) = (2 pi_hi - big_hi) + small_hi + lo parts;
        // 2 pi_hi - big_hi is exact (Sterbenz, big > pi), so no absolute error of
        // order ulp(2 pi) enters the small result
        const bool vbig = dh > 0.0f;
        const float bh = vbig ? va.x : aw.x, bl = vbig ? va.y : aw.y;
        const float sh = vbig ? aw.x : va.x, sl = vbig ? aw.y : va.y;
        d = ((kTwoPiHiF - bh) + sh) + ((kTwoPiLoF - bl) + sl);
    } else {
        d = fabsf(dh + (va.y - aw.y));
    }
    const float x = 0.5f * d;
    const float z = x * x;
    float t;
    if (x < 0.0078125f) {
        t = fmaf(z * x, -0.166666672f, x);
    } else {
        t = fmaf(z, -2.50521079e-08f, 2.75573188e-06f);
        t = fmaf(z, t, -1.98412701e-04f);
        t = fmaf(z, t, 8.33333377e-03f);
        t = fmaf(z, t, -1.66666672e-01f);
        t = fmaf(z * x, t, x);
    }
    const float ss = vb.x * w.z;  // 2 S_v S_w
    const float X = fmaf(ss * t, t, fmaf(va.z, w.y, va.w * w.x));
    const float err = fmaf(X, vb.z + w.w, fmaf(kC64 * vb.y, w.x + w.y, ss * t * kAngAbs));
    if (X + err <= 1.0f) return 1;
    if (X - err > 1.0f) return 0;
    return 2;
}

// asin(sqrt(Q)) for 0 <= Q < 1 (half the window angle), within 1e-6 relative:
// below sqrt(Q) = 1/8 the series y + y^3/6 + 3 y^5/40 (next term < 1.7e-7 y),
// else asinf; sqrt(Q) from rsqrtf (2 ulp).
__device__ __forceinline__ float half_angle(float Q)
{
    if (!(Q > 0.0f)) return 0.0f;
    const float y = Q * rsqrtf(Q);
    if (y < 0.125f) {
        const float y2 = y * y;
        return y * fmaf(y2, fmaf(y2, 0.075f, 0.16666667f), 1.0f);
    }
    return asinf(fminf(y, 1.0f));
}

// Window half-width in angle-key units (kFull: the whole band).  Filter mode,
// for band i with inner radius c' = c_i - kDeltaR: sin^2(theta/2) =
// (beta - cosh(r_v - c')/cosh R) / (2 sinh r_v sinh c' / cosh R), beta = 1 + the
// FP64 predicate's error bound for r_w < c_{i+1} + kDeltaR, all from the stored
// P, M, S with their error bounds added.
__device__ __forceinline__ uint32_t window_filter(const OwnerRegs &v, const BandShared &S, uint32_t i)
{
    const float Sc = S.S[i];
    if (i == 0 || !(Sc > 0.0f) || !(v.S2 > 0.0f)) return kFull;
    const float T = fmaf(v.P, S.Mm[i], v.M * S.P[i]);
    const float beta = fmaf(kC64 * v.PM, S.PMn[i], 1.0f);
    const float num = fmaf(1.0f + T, kWinE1, beta - T);
    const float den = v.S2 * Sc * (1.0f - (v.gam + 6.0f * kEps32));
    const float Q = __fdividef(num, den);  // 2 ulp, inside the final margin
    if (!(Q < 1.0f)) return kFull;
    const float th = half_angle(fmaxf(Q, 0.0f));
    const float keys = fmaf(th, kKeyPerRadF * (2.0f * (1.0f + 2e-5f)), 3.0f);
    return keys >= 2147483648.0f ? kFull : static_cast<uint32_t>(keys);
}

// Core half-width in angle-key units: every w of band i whose key is within it
// is an edge of the FP64 predicate.  X (exact, for the points' FP64 radii) must
// stay <= 1 - m at both band radii c' = c_i - dr and c'' = c_{i+1} + dr, with m =
// the predicate's rounding bound (plus kNearMargin); evaluated as lower bounds
// from the stored values.  Returns -1 for no core, kFull for the whole band.
__device__ __forceinline__ int64_t window_core(const OwnerRegs &v, const BandShared &S, uint32_t i)
{
    const float m = fmaf(kC64 * v.PM, S.PMn[i], kNearMargin);
    const float S2d = v.S2 * (1.0f + (v.gam + 6.0f * kEps32));
    float Q = 4.0f;
    // outer radius c''
    {
        const float T = fmaf(v.P, S.Mo[i], v.M * S.Po[i]);
        const float num = (1.0f - m - T) - (1.0f + T) * kWinE1;
        if (!(num > 0.0f)) return -1;
        const float den = S2d * S.So[i];
        if (den > 0.0f) Q = fminf(Q, __fdividef(num, den));
    }
    // inner radius c'
    {
        const float T = fmaf(v.P, S.Mm[i], v.M * S.P[i]);
        const float num = (1.0f - m - T) - (1.0f + T) * kWinE1;
        if (!(num > 0.0f)) return -1;
        const float den = S2d * S.S[i];
        if (den > 0.0f) Q = fminf(Q, __fdividef(num, den));
    }
    if (Q >= 1.0f) return kFull;
    // the series of half_angle is a lower bound of asin; the factor covers the
    // quotient's 2 ulp, rsqrtf and asinf
    const float th = half_angle(Q);
    const float keys = th * (kKeyPerRadF * (2.0f * (1.0f - 4e-5f))) - 4.0f;
    return keys < 0.0f ? -1 : static_cast<int64_t>(keys);
}

// FP64 mode window from the FP64 radius (Sec. III-B getMinMaxPhi), conservative
// for the rounded predicate: threshold (cosh R + 64 u cosh r_v cosh c_{i+1})(1 + 1e-12).
__device__ __forceinline__ uint32_t window_fp64(const OwnerRegs &v, const BandShared &S, uint32_t i, double coshR)
{
    const double ci = S.c[i];
    if (ci <= 0.0 || v.r <= 0.0 || v.sh <= 0.0) return kFull;
    constexpr double u = 0x1.0p-53;
    const double b = (coshR + 64.0 * u * v.ch * S.cosh_c[i + 1]) * (1.0 + 1e-12);
    const double Q = (b - ::cosh(v.r - ci)) / (2.0 * v.sh * S.sinh_c[i]);
    if (!(Q < 1.0)) return kFull;
    const double th = 2.0 * ::asin(::sqrt(Q > 0.0 ? Q : 0.0)) * (1.0 + 1e-9) + 1e-12;
    const double keys = th * kKeyPerRad + 3.0;
    return keys >= 2147483648.0 ? kFull : static_cast<uint32_t>(keys);
}

__device__ __forceinline__ uint32_t lower_key(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t x)
{
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ uint32_t upper_key(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t x)
{
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Four searches in one band through its bucket index ix (shift sh): each key's
// bucket gives the positions [ix[j], ix[j + 1]) that hold every key of that
// bucket, and a short bisection in lock step finishes.  r0 = first key >= x0,
// r1 = first key > x1, r2 = first key >= x2, r3 = first key > x3.
__device__ __forceinline__ void search4_indexed(const uint32_t *a, const uint32_t *ix, uint32_t sh, uint32_t x0,
                                                uint32_t x1, uint32_t x2, uint32_t x3, uint32_t &r0, uint32_t &r1,
                                                uint32_t &r2, uint32_t &r3)
{
    const uint32_t j0 = x0 >> sh, j1 = x1 >> sh, j2 = x2 >> sh, j3 = x3 >> sh;
    uint32_t l0 = __ldg(ix + j0), h0 = __ldg(ix + j0 + 1), l1 = __ldg(ix + j1), h1 = __ldg(ix + j1 + 1);
    uint32_t l2 = __ldg(ix + j2), h2 = __ldg(ix + j2 + 1), l3 = __ldg(ix + j3), h3 = __ldg(ix + j3 + 1);
    while (l0 < h0 || l1 < h1 || l2 < h2 || l3 < h3) {
        const uint32_t m0 = l0 + ((h0 - l0) >> 1), m1 = l1 + ((h1 - l1) >> 1);
        const uint32_t m2 = l2 + ((h2 - l2) >> 1), m3 = l3 + ((h3 - l3) >> 1);
        const uint32_t k0 = l0 < h0 ? __ldg(a + m0) : 0u, k1 = l1 < h1 ? __ldg(a + m1) : 0u;
        const uint32_t k2 = l2 < h2 ? __ldg(a + m2) : 0u, k3 = l3 < h3 ? __ldg(a + m3) : 0u;
        if (l0 < h0) { if (k0 < x0) l0 = m0 + 1; else h0 = m0; }
        if (l1 < h1) { if (k1 <= x1) l1 = m1 + 1; else h1 = m1; }
        if (l2 < h2) { if (k2 < x2) l2 = m2 + 1; else h2 = m2; }
        if (l3 < h3) { if (k3 <= x3) l3 = m3 + 1; else h3 = m3; }
    }
    r0 = l0;
    r1 = l1;
    r2 = l2;
    r3 = l3;
}

// Candidate positions in band [s, e) for keys in [a - W, a + W] (mod 2^32): at most
// two disjoint ranges [r0, r1) and [r2, r3).
__device__ __forceinline__ void key_ranges(const uint32_t *akey, uint32_t s, uint32_t e, uint32_t a, uint32_t W,
                                           uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    r2 = r3 = 0;
    if (W >= kFull) {
        r0 = s;
        r1 = e;
        return;
    }
    const uint32_t lo = a - W, hi = a + W;
    if (W <= a && hi >= a) {
        r0 = lower_key(akey, s, e, lo);
        r1 = upper_key(akey, s, e, hi);
    } else {  // wraps through 0: [lo, 2^32) and [0, hi]
        r0 = lower_key(akey, s, e, lo);
        r1 = e;
        r2 = s;
        r3 = upper_key(akey, s, e, hi);
    }
}

// tag = type (0 fringe, 1 core) | graph << 1 (batch)
template <bool kMulti>
__device__ __forceinline__ void push_heavy(const QueryArgs &a, Meta *C, uint32_t p, uint32_t lo, uint32_t hi,
                                           uint32_t tag)
{
    const uint32_t nch = (hi - lo + kChunk - 1) / kChunk;
    const uint32_t at = atomicAdd(&C->heavy_n, nch);
    if (at + nch > a.heavy_cap || at + nch < at) {
        atomicMax(&C->error, kErrListFull);
        return;
    }
    for (uint32_t j = 0; j < nch; ++j) {
        const uint32_t c0 = lo + j * kChunk;
        const uint32_t c1 = hi - c0 > kChunk ? c0 + kChunk : hi;
        a.heavy[at + j] = make_uint4(p, c0, c1, tag);
    }
}

template <bool kCsr>
__device__ __forceinline__ void write_edge(const QueryArgs &a, uint64_t pos, uint32_t i1, uint32_t i2)
{
    // streaming stores (evict first): the output is written once and must not
    // push the point arrays out of L2
    const uint32_t u = i1 < i2 ? i1 : i2, v = i1 < i2 ? i2 : i1;
    if (kCsr) {
        __stcs(reinterpret_cast<ulonglong2 *>(a.csr_keys) + pos,
               make_ulonglong2((static_cast<unsigned long long>(u) << 32) | v,
                               (static_cast<unsigned long long>(v) << 32) | u));
    } else {
        __stcs(reinterpret_cast<uint2 *>(a.pairs) + pos, make_uint2(u, v));
    }
}

// FP64 values of a point for the predicate (recheck and verification): the
// caller's point, or the sampler's FP64 point recomputed from its id.
__device__ __forceinline__ void fp64_point(const QueryArgs &a, const Meta *M, uint32_t id, double &ph, double &ch,
                                           double &sh)
{
    double r;
    if (a.src_phi) {
        ph = a.src_phi[id];
        r = a.src_r[id];
    } else {
        point_fp64(id, M->seed, M->R, M->cm1, M->inv_alpha, &ph, &r);
    }
    ch = dm::cosh(r);
    sh = dm::sinh(r);
}

// Verification mode: the FP64 predicate for a pair the filter or the core
// decided; a contradiction, or a decided pair within 1e-12 of the threshold, is
// counted.
__device__ __noinline__ void verify_pair(const QueryArgs &a, const Meta *Mg, Meta *C, uint32_t idv, uint32_t idw,
                                         int dec, double coshR)
{
    double pv, cv, sv, pw, cw, sw;
    fp64_point(a, Mg, idv, pv, cv, sv);
    fp64_point(a, Mg, idw, pw, cw, sw);
    const double L = predicate_L(pv, cv, sv, pw, cw, sw);
    if ((L <= coshR) != (dec == 1) || fabs(L - coshR) <= 1e-12 * coshR)
        atomicAdd(reinterpret_cast<unsigned long long *>(&C->verify_failures), 1ull);
}

// Decide candidate q (owner slot o); queue undecided pairs; in verification mode
// compare every decided pair with the FP64 predicate.
template <bool kFilter, bool kVerify>
__device__ __forceinline__ int decide(const QueryArgs &a, const Meta *Mg, Meta *C, const WarpSmem &W, uint32_t o,
                                      uint32_t q, bool in, double coshR, bool verify, uint64_t &near)
{
    const unsigned full = 0xffffffffu;
    int dec = 0;
    if (kFilter) {
        if (in) dec = filter_decide(W.oa[o], W.ob[o], a.P.ang[q], a.P.pms[q]);
        const uint32_t um = __ballot_sync(full, dec == 2);
        if (um) {
            const int lane = threadIdx.x & 31;
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&C->recheck_n, static_cast<uint32_t>(__popc(um)));
            base = __shfl_sync(full, base, 0);
            if (dec == 2) {
                const uint32_t at = base + __popc(um & ((1u << lane) - 1u));
                if (at < a.recheck_cap) a.recheck[at] = make_uint2(W.opos[o], q);
                else atomicMax(&C->error, kErrListFull);
            }
        }
        if (kVerify && verify && in && dec != 2) verify_pair(a, Mg, C, W.oid[o], a.P.id[q], dec, coshR);
    } else if (in) {
        const double2 v = W.od[o];
        const double chw = a.P.ch[q];
        const double L = predicate_L(v.x, v.y, W.osh[o], a.P.phi[q], chw, a.P.sh[q]);
        dec = L <= coshR;
        near += diag_count(L, coshR, v.y, chw);
    }
    return dec;
}

// Write a core chunk: owner idv and the sorted positions [q0, q0 + total), all
// certain edges; element j goes to base + j (coalesced), the id loads of
// kHeavyGroup 32-element windows issued together (one warp works a chunk on its
// own, so the loads in flight are what hides the memory latency).  Output: graph
// Mg's edge counter, its region starting at obase with room for cap pairs.
template <bool kCsr, bool kVerify>
__device__ __forceinline__ void write_core_chunk(const QueryArgs &a, Meta *Mg, Meta *C, uint64_t obase, uint64_t cap,
                                                 uint32_t idv, uint32_t q0, uint32_t total, double coshR, bool verify)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long *>(&Mg->m), total);
    base = __shfl_sync(full, base, 0);
    if (base + total > cap) return;
    base += obase;
    for (uint32_t j0 = 0; j0 < total; j0 += 32 * kHeavyGroup) {
        uint32_t w[kHeavyGroup];
#pragma unroll
        for (int g = 0; g < kHeavyGroup; ++g) {
            const uint32_t j = j0 + 32 * g + lane;
            w[g] = j < total ? __ldg(a.P.id + (q0 + j)) : 0u;
        }
#pragma unroll
        for (int g = 0; g < kHeavyGroup; ++g) {
            const uint32_t j = j0 + 32 * g + lane;
            if (j < total) {
                write_edge<kCsr>(a, base + j, idv, w[g]);
                if (kVerify && verify) verify_pair(a, Mg, C, idv, w[g], 1, coshR);
            }
        }
    }
}

// Decide, reserve and write the fringe stream of the queued entries [0, count),
// in segments of kBitWords rounds of 32 candidates: one decision bit per
// candidate, one output reservation per segment, then a replay of the set bits.
// The entry of a round's first candidate advances monotonically (warp-uniform);
// each lane then steps forward over the few entries its round crosses.
template <bool kFilter, bool kCsr, bool kVerify>
__device__ __forceinline__ void flush(const QueryArgs &a, Meta *Mg, Meta *C, uint64_t obase, uint64_t cap,
                                      WarpSmem &W, int count, double coshR, bool verify, uint64_t &near)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t total = W.pre[count];
    int e0 = 0;  // entry holding stream position j0
    for (uint32_t seg = 0; seg < total; seg += kBitWords * 32) {
        const uint32_t seg_end = total - seg > kBitWords * 32 ? seg + kBitWords * 32 : total;
        int words = 0;
        uint32_t edges = 0;
        for (uint32_t j0 = seg; j0 < seg_end; j0 += 32) {
            while (W.pre[e0 + 1] <= j0) ++e0;
            const uint32_t j = j0 + lane;
            const bool in = j < seg_end;
            int e = e0;
            if (in)
                while (W.pre[e + 1] <= j) ++e;
            const uint32_t q = W.lo[e] + (j - W.pre[e]);
            const int dec = decide<kFilter, kVerify>(a, Mg, C, W, W.own[e], q, in, coshR, verify, near);
            const uint32_t word = __ballot_sync(full, dec == 1);
            if (lane == 0) {
                W.bits[words] = word;
                W.round_entry[words] = static_cast<uint8_t>(e0);
            }
            ++words;
            edges += __popc(word);
        }
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0 && edges) base = atomicAdd(reinterpret_cast<unsigned long long *>(&Mg->m), edges);
        base = __shfl_sync(full, base, 0);
        if (edges && base + edges <= cap) {
            base += obase;
            uint32_t run = 0;
            for (int wi = 0; wi < words; ++wi) {
                const uint32_t word = W.bits[wi];
                if ((word >> lane) & 1u) {
                    const uint32_t j = seg + static_cast<uint32_t>(wi) * 32 + lane;
                    int e = W.round_entry[wi];
                    while (W.pre[e + 1] <= j) ++e;
                    const uint32_t q = W.lo[e] + (j - W.pre[e]);
                    write_edge<kCsr>(a, base + run + __popc(word & lt), W.oid[W.own[e]], a.P.id[q]);
                }
                run += __popc(word);
            }
        }
        __syncwarp();
    }
}

// Filter-mode fringe chunk of the owner in slot 0: candidates at the sorted
// positions [lo, lo + total) in rounds of 32, the candidate values of
// kFringeRounds rounds loaded together before they are tested; one decision bit
// per candidate, one output reservation per segment of kBitWords rounds, then a
// replay of the set bits (the id loads of kFringeRounds words issued together).
template <bool kCsr, bool kVerify>
__device__ __forceinline__ void test_fringe_chunk(const QueryArgs &a, Meta *Mg, Meta *C, uint64_t obase, uint64_t cap,
                                                  WarpSmem &W, uint32_t lo, uint32_t total, double coshR, bool verify)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const float4 va = W.oa[0], vb = W.ob[0];
    const uint32_t idv = W.oid[0], pv = W.opos[0];
    for (uint32_t seg = 0; seg < total; seg += kBitWords * 32) {
        const uint32_t seg_end = total - seg > kBitWords * 32 ? seg + kBitWords * 32 : total;
        int words = 0;
        uint32_t edges = 0;
        for (uint32_t j0 = seg; j0 < seg_end; j0 += 32 * kFringeRounds) {
            float2 ac[kFringeRounds];
            float4 pc[kFringeRounds];
#pragma unroll
            for (int r = 0; r < kFringeRounds; ++r) {
                const uint32_t j = j0 + 32 * r + lane;
                ac[r] = make_float2(0.0f, 0.0f);
                pc[r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (j < seg_end) {
                    ac[r] = a.P.ang[lo + j];
                    pc[r] = a.P.pms[lo + j];
                }
            }
#pragma unroll
            for (int r = 0; r < kFringeRounds; ++r) {
                if (j0 + 32 * r >= seg_end) break;  // warp-uniform
                const uint32_t j = j0 + 32 * r + lane;
                const bool in = j < seg_end;
                const int dec = in ? filter_decide(va, vb, ac[r], pc[r]) : 0;
                const uint32_t um = __ballot_sync(full, dec == 2);
                if (um) {
                    uint32_t rb = 0;
                    if (lane == 0) rb = atomicAdd(&C->recheck_n, static_cast<uint32_t>(__popc(um)));
                    rb = __shfl_sync(full, rb, 0);
                    if (dec == 2) {
                        const uint32_t at = rb + __popc(um & lt);
                        if (at < a.recheck_cap) a.recheck[at] = make_uint2(pv, lo + j);
                        else atomicMax(&C->error, kErrListFull);
                    }
                }
                if (kVerify && verify && in && dec != 2) verify_pair(a, Mg, C, idv, a.P.id[lo + j], dec, coshR);
                const uint32_t word = __ballot_sync(full, dec == 1);
                if (lane == 0) W.bits[words] = word;
                ++words;
                edges += __popc(word);
            }
        }
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0 && edges) base = atomicAdd(reinterpret_cast<unsigned long long *>(&Mg->m), edges);
        base = __shfl_sync(full, base, 0);
        if (edges && base + edges <= cap) {
            base += obase;
            uint32_t run = 0;
            for (int w0 = 0; w0 < words; w0 += kFringeRounds) {
                uint32_t word[kFringeRounds], idw[kFringeRounds];
#pragma unroll
                for (int r = 0; r < kFringeRounds; ++r) {
                    word[r] = w0 + r < words ? W.bits[w0 + r] : 0u;
                    idw[r] = 0u;
                    if ((word[r] >> lane) & 1u)
                        idw[r] = __ldg(a.P.id + (lo + seg + static_cast<uint32_t>(w0 + r) * 32 + lane));
                }
#pragma unroll
                for (int r = 0; r < kFringeRounds; ++r) {
                    if ((word[r] >> lane) & 1u) write_edge<kCsr>(a, base + run + __popc(word[r] & lt), idv, idw[r]);
                    run += __popc(word[r]);
                }
            }
        }
        __syncwarp();
    }
}

// Per-warp shared state of the batch kernel.  For each band the 32 lanes' tested
// pieces are laid end to end as the fringe stream (lane after lane).  own[]
// tabulates the owner lane of kOwn consecutive stream elements, one byte each, so
// that a lane finds the owner of any element with one shared-memory load; the
// owners' values are read from fr / oid / oa / ob (or od / osh in FP64 mode).  The
// core pieces need no table: they are written lane-major.
constexpr uint32_t kOwn = 1024;       // stream elements whose owners are tabulated at once
constexpr int kMaxFringe = 64;        // fringe candidates a lane keeps (two pieces of at most 32)
constexpr uint32_t kAccCap = 128;     // accepted fringe pairs a warp keeps per band

template <bool kFilter, uint32_t kAcc>
struct BatchSmem {
    uint32_t own[kOwn / 4];                  // owner lane of stream element j0 + e: byte e
    uint32_t bits[32 * kMaxFringe / 32];     // fringe decisions, bit j of word j / 32
    uint4 fr[32];                            // lane's fringe: stream start, f0, length of [f0, f1), f2
    uint32_t oid[32];                        // lane's vertex id
    uint2 acc[kAcc ? kAcc : 1];              // accepted fringe pairs (owner id, candidate id), stream order
    float4 oa[kFilter ? 32 : 1], ob[kFilter ? 32 : 1];  // filter values (as load_owner stores them)
    double2 od[kFilter ? 1 : 32];            // FP64 mode: phi, cosh r
    double osh[kFilter ? 1 : 32];            // FP64 mode: sinh r
};

// A warp's shared memory in the batch kernel, at least the size of WarpSmem:
// without kept fringe pairs, padding BatchSmem to that size made the batched
// range query (persistent launch) 11.9 instead of 12.6 ms for the 4096-graph
// workload.  With 128 kept pairs BatchSmem is the larger; the persistent
// kernel's shared memory (65 KB) still leaves room for 3 CTAs per SM.
template <bool kFilter, uint32_t kAcc>
union PerWarp {
    BatchSmem<kFilter, kAcc> b;
    WarpSmem unused;
};

// own bytes of the stream elements [j0, j0 + kOwn) inside [s, s + len) := lane.
__device__ __forceinline__ void fill_owner(uint32_t *own, uint32_t j0, uint32_t s, uint32_t len, uint32_t lane)
{
    const uint32_t e = s + len;
    uint32_t a = s > j0 ? s - j0 : 0u;
    uint32_t b = e > j0 ? e - j0 : 0u;
    if (b > kOwn) b = kOwn;
    uint8_t *o = reinterpret_cast<uint8_t *>(own);
    const uint32_t rep = lane * 0x01010101u;
    while (a < b && (a & 3u)) o[a++] = static_cast<uint8_t>(lane);
    while (a + 4 <= b) {
        own[a >> 2] = rep;
        a += 4;
    }
    while (a < b) o[a++] = static_cast<uint8_t>(lane);
}

__device__ __forceinline__ uint32_t owner_of(const uint32_t *own, uint32_t e)
{
    return reinterpret_cast<const uint8_t *>(own)[e];
}

// Sorted position of fringe stream element j (owner values r = fr[owner]).
__device__ __forceinline__ uint32_t fringe_pos(uint4 r, uint32_t j)
{
    const uint32_t t = j - r.x;
    return t < r.z ? r.y + t : r.w + (t - r.z);
}

// Decide fringe stream element j (owner lane L at sorted position p, candidate q):
// 1 = edge, 0 = no edge, 2 = undecided (queued for the FP64 recheck).
template <bool kFilter, bool kVerify, class WS>
__device__ __forceinline__ int decide_stream(const QueryArgs &a, const Meta *Mg, Meta *C, const WS &W,
                                             uint32_t L, uint32_t p, uint32_t q, bool in, double coshR, bool verify,
                                             uint64_t &near)
{
    const unsigned full = 0xffffffffu;
    int dec = 0;
    if (kFilter) {
        if (in) dec = filter_decide(W.oa[L], W.ob[L], a.P.ang[q], a.P.pms[q]);
        const uint32_t um = __ballot_sync(full, dec == 2);
        if (um) {
            const int lane = threadIdx.x & 31;
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&C->recheck_n, static_cast<uint32_t>(__popc(um)));
            base = __shfl_sync(full, base, 0);
            if (dec == 2) {
                const uint32_t at = base + __popc(um & ((1u << lane) - 1u));
                if (at < a.recheck_cap) a.recheck[at] = make_uint2(p, q);
                else atomicMax(&C->error, kErrListFull);
            }
        }
        if (kVerify && verify && in && dec != 2) verify_pair(a, Mg, C, W.oid[L], a.P.id[q], dec, coshR);
    } else if (in) {
        const double2 v = W.od[L];
        const double chw = a.P.ch[q];
        const double Lv = predicate_L(v.x, v.y, W.osh[L], a.P.phi[q], chw, a.P.sh[q]);
        dec = Lv <= coshR;
        near += diag_count(Lv, coshR, v.y, chw);
    }
    return dec;
}

// One warp per batch of 32 consecutive sorted points, lane = point.  For each band
// every lane computes its window and core (Sec. III-B) and the candidate pieces;
// the warp decides the fringe stream 32 candidates at a time (all lanes busy
// whatever the split between the lanes), reserves the band's edges with one
// atomic add, and writes the core pieces (lane-major) and the fringe edges (in
// stream order) as contiguous blocks.
// kMulti (a batch of graphs): batches are 32-point slices of the tiles, each warp
// keeps the band table of its current graph in its own shared memory, and edges
// go to the graph's output region and counter; lists and work counters live in
// the control block.
template <bool kFilter, bool kCsr, bool kMulti, bool kVerify>
__device__ __forceinline__ void batch_body(const QueryArgs &a, BandShared *Sm, PerWarp<kFilter, kAccCap> *Wsm)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    BandShared &S = Sm[kMulti ? (threadIdx.x >> 5) : 0];
    auto &W = Wsm[threadIdx.x >> 5].b;
    constexpr uint32_t kAcc = kAccCap;
    Meta *C = kMulti ? a.M + a.bt.G : a.M;  // counters and lists
    Meta *M = a.M;                          // the current graph
    if (!kMulti) {
        load_bands(S, M);
        __syncthreads();
        if (M->error || (M->filter != 0) != kFilter) return;
    } else if (C->error) {
        return;
    }
    const unsigned full = 0xffffffffu;
    const uint32_t n = static_cast<uint32_t>(a.P.n);
    uint32_t B = M->B;
    double coshR = M->coshR;
    bool verify = kVerify && M->verify != 0;  // the variant without verification has no checks at all
    uint64_t obase = 0, cap = a.capacity;  // output region of the current graph
    uint32_t cur_g = 0xffffffffu;
    bool skip = false;
    const uint32_t nbatch = kMulti ? a.bt.num_tiles * (kTilePoints / 32)
                                   : (a.batch_hi ? a.batch_hi - a.batch_lo : (n + 31) / 32);
    unsigned long long cand = 0;
    uint64_t near = 0;
    // batches in sorted order from kClaimCounters interleaved counters (counter c
    // hands out batches c, c + kClaimCounters, ...): the costly inner-band batches
    // start first and the rest fill in around them.  A warp starts on its own
    // counter and moves to the next one when it is used up; it stops when all are.
    uint32_t ci = (blockIdx.x * kWarps + (threadIdx.x >> 5)) % kClaimCounters, misses = 0;
    for (;;) {
        uint32_t batch = 0;
        if (lane == 0) batch = atomicAdd(&C->claim[ci * 32], 1u) * kClaimCounters + ci;
        batch = __shfl_sync(full, batch, 0);
        if (batch >= nbatch) {
            if (++misses == kClaimCounters) break;
            ci = ci + 1 == kClaimCounters ? 0 : ci + 1;
            continue;
        }
        misses = 0;
        uint32_t p0, cnt;  // first sorted position and points of this batch
        if (kMulti) {
            const uint4 T = a.bt.tiles[batch / (kTilePoints / 32)];
            const uint32_t sub = (batch % (kTilePoints / 32)) * 32;
            if (sub >= T.z) continue;
            if (T.x != cur_g) {
                cur_g = T.x;
                M = a.M + cur_g;
                __syncwarp();
                load_bands_from(S, M, lane, 32);
                __syncwarp();
                B = M->B;
                coshR = M->coshR;
                verify = kVerify && M->verify != 0;
                obase = a.bt.out_off[cur_g];
                cap = a.bt.out_off[cur_g + 1] - obase;
                skip = M->error || (M->filter != 0) != kFilter;
            }
            if (skip) continue;
            p0 = T.y + sub;
            cnt = T.z - sub < 32 ? T.z - sub : 32;
        } else {
            p0 = (a.batch_lo + batch) * 32;
            cnt = n - p0 < 32 ? n - p0 : 32;
        }
        const uint32_t p = p0 + lane;
        const bool valid = static_cast<uint32_t>(lane) < cnt;
        OwnerRegs mine{};
        uint32_t bv = B, akv = 0, idv = 0;
        __syncwarp();  // the previous batch's readers of W are done
        if (valid) {
            idv = a.P.id[p];
            bv = static_cast<uint32_t>(a.P.key[p] >> 32);
            akv = a.P.akey[p];
            if (kFilter) {
                const float2 an = a.P.ang[p];
                const float4 q = a.P.pms[p];
                mine.P = q.x;
                mine.M = q.y;
                mine.S2 = 2.0f * q.z;
                mine.PM = q.x + q.y;
                mine.gam = q.w;
                W.oa[kFilter ? lane : 0] = make_float4(an.x, an.y, q.x, q.y);
                W.ob[kFilter ? lane : 0] = make_float4(mine.S2, mine.PM, kCBase + q.w, 0.0f);
            } else {
                mine.r = a.P.r[p];
                mine.ch = a.P.ch[p];
                mine.sh = a.P.sh[p];
                W.od[kFilter ? 0 : lane] = make_double2(a.P.phi[p], mine.ch);
                W.osh[kFilter ? 0 : lane] = mine.sh;
            }
        }
        const uint32_t bmin = __reduce_min_sync(full, bv);
        uint32_t kept = 0;  // candidates this batch keeps (warp-uniform)
        for (uint32_t i = bmin; i < B; ++i) {
            const uint32_t s = S.start[i], e = S.start[i + 1];
            if (s == e) continue;
            const bool active = valid && i >= bv;
            uint32_t Wf = 0;
            int64_t Wc = -1;
            bool plain = false;  // window lies inside [0, 2^32): union search and core allowed
            if (active) {
                Wf = kFilter ? window_filter(mine, S, i) : window_fp64(mine, S, i, coshR);
                plain = Wf < kFull && Wf <= akv && akv + Wf >= akv;
                if (kFilter && plain) Wc = window_core(mine, S, i);
            }
            // pieces: fringe [f0, f1), core [c0, c1), fringe [f2, f3)
            uint32_t f0 = 0, f1 = 0, f2 = 0, f3 = 0, c0 = 0, c1 = 0;
            if (active) {
                if (plain) {
                    const uint32_t wc = Wc < 0 ? 0u : (Wc >= static_cast<int64_t>(Wf) ? Wf : static_cast<uint32_t>(Wc));
                    search4_indexed(a.P.akey, a.bidx + S.ioff[i], S.ishift[i], akv - Wf, akv + Wf, akv - wc, akv + wc,
                                    f0, f3, c0, c1);
                    if (Wc < 0) {  // no core: the fringe is the whole window
                        c0 = c1 = 0;
                        f1 = f3;
                        f2 = f3;
                    } else {
                        f1 = c0;
                        f2 = c1;
                    }
                } else {
                    key_ranges(a.P.akey, s, e, akv, Wf, f0, f1, f2, f3);
                }
                if (i == bv) {  // same band: each pair once, from the smaller position
                    const uint32_t m1 = p + 1;
                    f0 = f0 > m1 ? f0 : m1;
                    f2 = f2 > m1 ? f2 : m1;
                    c0 = c0 > m1 ? c0 : m1;
                }
                if (f1 < f0) f1 = f0;
                if (f3 < f2) f3 = f2;
                if (c1 < c0) c1 = c0;
                cand += (f1 - f0) + (f3 - f2) + (c1 - c0);
                // a lane keeps at most fringe_limit (<= 32) candidates of each of its
                // two fringe pieces; a batch keeps about the budget's candidates;
                // longer ranges become chunks that every warp shares
                const uint32_t room = kept < S.budget ? (S.budget - kept) / 32 : 0;
                const uint32_t hc = S.core_heavy < (room > 64 ? room : 64) ? S.core_heavy : (room > 64 ? room : 64);
                const uint32_t gtag = kMulti ? cur_g << 1 : 0u;
                if (f1 - f0 > S.fringe_limit) {
                    push_heavy<kMulti>(a, C, p, f0, f1, gtag);
                    f1 = f0;
                }
                if (f3 - f2 > S.fringe_limit) {
                    push_heavy<kMulti>(a, C, p, f2, f3, gtag);
                    f3 = f2;
                }
                if (c1 - c0 > hc) {
                    push_heavy<kMulti>(a, C, p, c0, c1, gtag | 1u);
                    c1 = c0;
                }
            }
            const uint32_t nl = f1 - f0, nf = nl + (f3 - f2), nc = c1 - c0;
            uint32_t fi = nf;  // inclusive scan over the lanes
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(full, fi, off);
                if (lane >= off) fi += y;
            }
            const uint32_t F = __shfl_sync(full, fi, 31), T = __reduce_add_sync(full, nc);
            if (F + T == 0) continue;
            const uint32_t fs = fi - nf;  // the lane's fringe stream start
            __syncwarp();  // the previous band's readers of W are done
            W.fr[lane] = make_uint4(fs, f0, nl, f2);
            W.oid[lane] = idv;
            // 1. the fringe stream, 32 candidates per step: one decision bit each; the
            // candidate's id is loaded with its values, and the first kAcc accepted
            // pairs are kept in stream order
            uint32_t nfe = 0;
            for (uint32_t j0 = 0; j0 < F; j0 += kOwn) {
                fill_owner(W.own, j0, fs, nf, lane);
                __syncwarp();
                const uint32_t jend = F - j0 > kOwn ? j0 + kOwn : F;
                for (uint32_t jw = j0; jw < jend; jw += 32) {
                    const uint32_t j = jw + lane;
                    const bool in = j < jend;
                    uint32_t L = 0, q = 0, idw = 0;
                    if (in) {
                        L = owner_of(W.own, j - j0);
                        q = fringe_pos(W.fr[L], j);
                        if (kAcc) idw = __ldg(a.P.id + q);
                    }
                    const int dec = decide_stream<kFilter, kVerify>(a, M, C, W, L, p0 + L, q, in, coshR, verify, near);
                    const uint32_t word = __ballot_sync(full, dec == 1);
                    if (lane == 0) W.bits[jw >> 5] = word;
                    if (kAcc && dec == 1) {
                        const uint32_t at = nfe + __popc(word & lt);
                        if (at < kAcc) W.acc[at] = make_uint2(W.oid[L], idw);
                    }
                    nfe += __popc(word);
                }
                __syncwarp();
            }
            // one reservation for the band's edges: [base, base + T) holds the core
            // edges, then come the fringe edges in stream order
            const uint32_t total = T + nfe;
            kept += total;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long *>(&M->m), total);
            base = __shfl_sync(full, base, 0);
            if (base + total > cap) continue;
            base += obase;
            // 2. the fringe edges: from the kept pairs when all fit, else by a replay
            // of the decision bits (the owner table still holds the last fringe chunk)
            if (kAcc && nfe && nfe <= kAcc) {
                for (uint32_t e = lane; e < nfe; e += 32) {
                    const uint2 v = W.acc[e];
                    write_edge<kCsr>(a, base + T + e, v.x, v.y);
                }
            } else if (nfe) {
                uint64_t pos = base + T;
                for (uint32_t j0 = 0; j0 < F; j0 += kOwn) {
                    if (F > kOwn) {
                        __syncwarp();
                        fill_owner(W.own, j0, fs, nf, lane);
                        __syncwarp();
                    }
                    const uint32_t jend = F - j0 > kOwn ? j0 + kOwn : F;
                    for (uint32_t jw = j0; jw < jend; jw += 32) {
                        const uint32_t word = W.bits[jw >> 5];
                        if ((word >> lane) & 1u) {
                            const uint32_t j = jw + lane;
                            const uint32_t L = owner_of(W.own, j - j0);
                            const uint32_t q = fringe_pos(W.fr[L], j);
                            write_edge<kCsr>(a, pos + __popc(word & lt), W.oid[L], __ldg(a.P.id + q));
                        }
                        pos += __popc(word);
                    }
                }
            }
            // 3. the core pieces, lane-major: step t writes the t-th element of every
            // lane's piece.  While every lane has one (t below the shortest piece)
            // they go to base + 32 t + lane, kCoreUnroll steps with their id loads
            // issued together; past it the lanes that still have one are ranked by
            // a ballot.  No owner lookup per element, and every step's stores are
            // contiguous.
            {
                const uint32_t mn = __reduce_min_sync(full, nc), mx = __reduce_max_sync(full, nc);
                const uint32_t *idp = a.P.id + c0;
                uint32_t t = 0;
                for (; t + kCoreUnroll <= mn; t += kCoreUnroll) {
                    uint32_t w[kCoreUnroll];
#pragma unroll
                    for (int g = 0; g < kCoreUnroll; ++g) w[g] = __ldg(idp + t + g);
#pragma unroll
                    for (int g = 0; g < kCoreUnroll; ++g) {
                        write_edge<kCsr>(a, base + static_cast<uint64_t>(t + g) * 32u + lane, idv, w[g]);
                        if (kVerify && verify) verify_pair(a, M, C, idv, w[g], 1, coshR);
                    }
                }
                for (; t < mn; ++t) {
                    const uint32_t w = __ldg(idp + t);
                    write_edge<kCsr>(a, base + static_cast<uint64_t>(t) * 32u + lane, idv, w);
                    if (kVerify && verify) verify_pair(a, M, C, idv, w, 1, coshR);
                }
                uint64_t pos = base + static_cast<uint64_t>(mn) * 32u;
                for (; t < mx; ++t) {
                    const bool act = t < nc;
                    const uint32_t m = __ballot_sync(full, act);
                    if (act) {
                        const uint32_t w = __ldg(idp + t);
                        write_edge<kCsr>(a, pos + __popc(m & lt), idv, w);
                        if (kVerify && verify) verify_pair(a, M, C, idv, w, 1, coshR);
                    }
                    pos += __popc(m);
                }
            }
        }
    }
    for (int off = 16; off; off >>= 1) cand += __shfl_down_sync(full, cand, off);
    if (lane == 0 && cand) atomicAdd(reinterpret_cast<unsigned long long *>(&C->candidates), cand);
    flush_diag(C, near);
}

template <bool kFilter, bool kCsr, bool kMulti, bool kVerify>
__global__ void __launch_bounds__(kThreads, kBatchMinBlocks) batch_kernel(QueryArgs a)
{
    __shared__ BandShared Sm[kMulti ? kWarps : 1];
    __shared__ PerWarp<kFilter, kAccCap> Wsm[kWarps];
    batch_body<kFilter, kCsr, kMulti, kVerify>(a, Sm, Wsm);
}

// One heavy chunk h (a record of the chunk list) by one warp: at most kChunk
// candidates of one owner, tested (type 0) or a core chunk of certain edges
// (type 1); w = type | graph << 1 (graph 0 for a single graph).
template <bool kFilter, bool kCsr, bool kMulti, bool kVerify>
__device__ __forceinline__ void heavy_item(const QueryArgs &a, Meta *C, WarpSmem &W, uint4 h, uint64_t &near)
{
    const int lane = threadIdx.x & 31;
    const uint32_t tag = h.w;
    const uint32_t g = tag >> 1;
    Meta *Mg = kMulti ? a.M + g : a.M;
    if (kMulti && (Mg->error || (Mg->filter != 0) != kFilter)) return;
    const double coshR = Mg->coshR;
    const bool verify = kVerify && Mg->verify != 0;
    const uint64_t obase = kMulti ? a.bt.out_off[g] : 0;
    const uint64_t cap = kMulti ? a.bt.out_off[g + 1] - obase : a.capacity;
    const bool core = (tag & 1u) != 0;
    if (lane == 0) {
        load_owner<kFilter>(a.P, W, 0, h.x);
        if (!core) {
            W.lo[0] = h.y;
            W.pre[0] = 0;
            W.pre[1] = h.z - h.y;
            W.own[0] = 0;
        }
    }
    __syncwarp();
    if (core) write_core_chunk<kCsr, kVerify>(a, Mg, C, obase, cap, W.oid[0], h.y, h.z - h.y, coshR, verify);
    else if (kFilter) test_fringe_chunk<kCsr, kVerify>(a, Mg, C, obase, cap, W, h.y, h.z - h.y, coshR, verify);
    else flush<kFilter, kCsr, kVerify>(a, Mg, C, obase, cap, W, 1, coshR, verify, near);
    __syncwarp();
}

// Heavy chunks: one warp per chunk, round robin over the warps (all chunks hold
// at most kChunk candidates and most hold exactly that): no claim traffic on a
// shared counter.  A phased query starts after the chunks of its earlier phases.
template <bool kFilter, bool kCsr, bool kMulti, bool kVerify>
__device__ __forceinline__ void heavy_body(const QueryArgs &a, WarpSmem *Wsm)
{
    Meta *C = kMulti ? a.M + a.bt.G : a.M;
    if (C->error || (!kMulti && (C->filter != 0) != kFilter)) return;
    const int warp = threadIdx.x >> 5;
    WarpSmem &W = Wsm[warp];
    const uint32_t count = C->heavy_n < a.heavy_cap ? C->heavy_n : a.heavy_cap;
    const uint32_t start = C->heavy_lo;
    uint64_t near = 0;
    const uint32_t gwarps = gridDim.x * kWarps;
    for (uint32_t item = start + blockIdx.x * kWarps + warp; item < count; item += gwarps)
        heavy_item<kFilter, kCsr, kMulti, kVerify>(a, C, W, a.heavy[item], near);
    flush_diag(C, near);
}

template <bool kFilter, bool kCsr, bool kMulti, bool kVerify>
__global__ void __launch_bounds__(kThreads) heavy_kernel(QueryArgs a)
{
    __shared__ WarpSmem Wsm[kWarps];
    heavy_body<kFilter, kCsr, kMulti, kVerify>(a, Wsm);
}

// FP64 recheck of the pairs the filter left undecided: the predicate of Eq. 3 on
// the FP64 points, and the edges appended with one reservation per warp.
template <bool kCsr>
__global__ void __launch_bounds__(kThreads) recheck_kernel(QueryArgs a)
{
    Meta *M = a.M;
    if (M->error || !M->filter) return;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t count = M->recheck_n < a.recheck_cap ? M->recheck_n : a.recheck_cap;
    const double coshR = M->coshR;
    uint64_t near = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t w0 = M->recheck_lo + ((blockIdx.x * blockDim.x + threadIdx.x) & ~31u); w0 < count; w0 += stride) {
        const uint32_t idx = w0 + lane;
        bool edge = false;
        uint32_t idv = 0, idw = 0;
        if (idx < count) {
            const uint2 pq = a.recheck[idx];
            idv = a.P.id[pq.x];
            idw = a.P.id[pq.y];
            double pv, cv, sv, pw, cw, sw;
            fp64_point(a, M, idv, pv, cv, sv);
            fp64_point(a, M, idw, pw, cw, sw);
            const double L = predicate_L(pv, cv, sv, pw, cw, sw);
            edge = L <= coshR;
            near += diag_count(L, coshR, cv, cw);
        }
        const uint32_t word = __ballot_sync(full, edge);
        if (!word) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long *>(&M->m), __popc(word));
        base = __shfl_sync(full, base, 0);
        if (edge && base + __popc(word) <= a.capacity) write_edge<kCsr>(a, base + __popc(word & lt), idv, idw);
    }
    flush_diag(M, near);
    if (blockIdx.x == 0 && threadIdx.x == 0) M->rechecks = count;
}

// Batch recheck: each pair's graph from the owner position; one output slot per
// edge from the graph's counter (the pairs are few).  Grid-stride over the list.
__device__ __forceinline__ void recheck_batch_body(const QueryArgs &a)
{
    Meta *C = a.M + a.bt.G;
    if (C->error) return;
    const uint32_t count = C->recheck_n < a.recheck_cap ? C->recheck_n : a.recheck_cap;
    uint64_t near = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += stride) {
        const uint2 pq = a.recheck[idx];
        uint32_t lo = 0, hi = a.bt.G;  // graph g: pt_off[g] <= pq.x < pt_off[g + 1]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.bt.pt_off[mid] <= pq.x) lo = mid;
            else hi = mid;
        }
        Meta *Mg = a.M + lo;
        const uint32_t idv = a.P.id[pq.x], idw = a.P.id[pq.y];
        double pv, cv, sv, pw, cw, sw;
        fp64_point(a, Mg, idv, pv, cv, sv);
        fp64_point(a, Mg, idw, pw, cw, sw);
        const double coshR = Mg->coshR;
        const double L = predicate_L(pv, cv, sv, pw, cw, sw);
        near += diag_count(L, coshR, cv, cw);
        if (L <= coshR) {
            const unsigned long long at = atomicAdd(reinterpret_cast<unsigned long long *>(&Mg->m), 1ull);
            const uint64_t obase = a.bt.out_off[lo];
            if (at < a.bt.out_off[lo + 1] - obase) write_edge<false>(a, obase + at, idv, idw);
        }
    }
    flush_diag(C, near);
    if (blockIdx.x == 0 && threadIdx.x == 0) C->rechecks = count;
}

// Between the filter and the FP64 phase of a batch: the work counters and the
// heavy list start again (the recheck list and the statistics carry over).
__device__ __forceinline__ void reset_phase(Meta *C)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        C->work_counter = 0;
        for (uint32_t c = 0; c < kClaimCounters; ++c) C->claim[c * 32] = 0;
        C->heavy_n = 0;
        C->heavy_next = 0;
    }
}


// End of phase p of a phased query: its edges are final, the next phase starts its
// claims, chunks and rechecks after the ones done.
__global__ void phase_end_kernel(Meta *M, uint32_t p, uint32_t heavy_cap, uint32_t recheck_cap, uint64_t *host_m)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t m = M->m;
    M->m_phase[p] = m;
    for (uint32_t c = 0; c < kClaimCounters; ++c) M->claim[c * 32] = 0;
    M->heavy_lo = M->heavy_n < heavy_cap ? M->heavy_n : heavy_cap;
    M->recheck_lo = M->recheck_n < recheck_cap ? M->recheck_n : recheck_cap;
    if (host_m) {
        *reinterpret_cast<volatile uint64_t *>(host_m + p) = m;
        __threadfence_system();
    }
}

// ------------------------------------------------------------------ subset query
// Neighbours of the moved vertices (dynamic model, Sec. III-C), for the update of
// an edge list: moved vertex v (sorted position owners[j]) against every
// band, inward and outward (the window of Sec. III-B at the band's inner radius
// bounds every band).  A pair (v, w) counts when w is not v and either w did not
// move or id_v < id_w (a pair of two moved vertices once).  Filter mode decides
// undecided pairs with the FP64 predicate on the spot; FP64 mode tests every
// candidate with it.  kEmit = false writes the count of vertex j; kEmit = true
// writes its pairs from *base + offsets[j] (pairs past the capacity are skipped).
constexpr uint32_t kSubsetPiece = 64;     // longer pieces become chunks
constexpr uint32_t kSubsetChunk = 4096;   // candidates per chunk

struct SubsetArgs {
    const uint32_t *owners;
    uint64_t count;                          // moved vertices; counts / offsets slots 0 .. count - 1
    const unsigned long long *owners_found;  // owners listed on the device (<= count when ids repeat)
    uint4 *chunks;                           // {owner index, lo, hi, certain}; slots count + c
    uint64_t chunk_cap;
    unsigned long long *chunk_n;
    const uint8_t *moved_by_pos;
    uint32_t *counts;
    const uint64_t *offsets;
    const unsigned long long *base;
    uint64_t capacity;
};

// The pair (v at sorted position p, w at q).  Filter mode: the FP32 filter, and
// the FP64 predicate (both points recomputed) when it cannot decide.
template <bool kFilter>
__device__ __forceinline__ bool subset_test(const QueryArgs &a, const Meta *M, float4 va, float4 vb, uint32_t p,
                                            uint32_t q, double coshR)
{
    if (kFilter) {
        const int dec = filter_decide(va, vb, a.P.ang[q], a.P.pms[q]);
        if (dec != 2) return dec == 1;
        double pv, cv, sv, pw, cw, sw;
        fp64_point(a, M, a.P.id[p], pv, cv, sv);
        fp64_point(a, M, a.P.id[q], pw, cw, sw);
        return predicate_L(pv, cv, sv, pw, cw, sw) <= coshR;
    }
    return predicate_L(a.P.phi[p], a.P.ch[p], a.P.sh[p], a.P.phi[q], a.P.ch[q], a.P.sh[q]) <= coshR;
}

// One thread per (moved vertex, band): slot t = j * B + i of counts / offsets.
// Its pairs are written contiguously from its offset.
template <bool kFilter, bool kEmit>
__global__ void __launch_bounds__(kThreads) subset_kernel(QueryArgs a, SubsetArgs sa)
{
    __shared__ BandShared S;
    Meta *M = a.M;
    load_bands(S, M);
    __syncthreads();
    if (M->error || (M->filter != 0) != kFilter) return;
    const uint32_t B = M->B;
    const double coshR = M->coshR;
    const uint64_t found_n = *sa.owners_found < sa.count ? *sa.owners_found : sa.count;
    const uint64_t slots = sa.count * B;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < slots; t += stride) {
        const uint64_t j = t / B;
        const uint32_t i = static_cast<uint32_t>(t - j * B);
        const uint32_t s = S.start[i], e = S.start[i + 1];
        if (j >= found_n || s == e) {  // not listed, or an empty band: no pairs
            if (!kEmit) sa.counts[t] = 0;
            continue;
        }
        const uint32_t p = sa.owners[j];
        const uint32_t idv = a.P.id[p];
        const uint32_t akv = a.P.akey[p];
        OwnerRegs mine{};
        float4 va = make_float4(0, 0, 0, 0), vb = va;
        if (kFilter) {
            const float2 an = a.P.ang[p];
            const float4 q = a.P.pms[p];
            mine.P = q.x;
            mine.M = q.y;
            mine.S2 = 2.0f * q.z;
            mine.PM = q.x + q.y;
            mine.gam = q.w;
            va = make_float4(an.x, an.y, q.x, q.y);
            vb = make_float4(mine.S2, mine.PM, kCBase + q.w, 0.0f);
        } else {
            mine.r = a.P.r[p];
            mine.ch = a.P.ch[p];
            mine.sh = a.P.sh[p];
        }
        uint64_t out = 0;
        if (kEmit) out = *sa.base + sa.offsets[t];
        uint32_t found = 0;
        const uint32_t Wf = kFilter ? window_filter(mine, S, i) : window_fp64(mine, S, i, coshR);
        const bool plain = Wf < kFull && Wf <= akv && akv + Wf >= akv;
        uint32_t f0, f1, f2, f3, c0 = 0, c1 = 0;
        if (plain) {
            int64_t Wc = -1;
            if (kFilter) Wc = window_core(mine, S, i);
            const uint32_t wc = Wc < 0 ? 0u : (Wc >= static_cast<int64_t>(Wf) ? Wf : static_cast<uint32_t>(Wc));
            search4_indexed(a.P.akey, a.bidx + S.ioff[i], S.ishift[i], akv - Wf, akv + Wf, akv - wc, akv + wc, f0,
                            f3, c0, c1);
            if (Wc < 0) {
                c0 = c1 = f3;
                f1 = f2 = f3;
            } else {
                f1 = c0;
                f2 = c1;
            }
        } else {
            key_ranges(a.P.akey, s, e, akv, Wf, f0, f1, f2, f3);
        }
        // three pieces: [f0, f1) and [f2, f3) tested, [c0, c1) certain; long
        // pieces go to the chunk list (once, in the counting pass)
        for (int piece = 0; piece < 3; ++piece) {
            const uint32_t lo = piece == 0 ? f0 : (piece == 1 ? c0 : f2);
            const uint32_t hi = piece == 0 ? f1 : (piece == 1 ? c1 : f3);
            if (hi > lo && hi - lo > kSubsetPiece) {
                if (!kEmit) {
                    const uint32_t nc = (hi - lo + kSubsetChunk - 1) / kSubsetChunk;
                    const unsigned long long at = atomicAdd(sa.chunk_n, static_cast<unsigned long long>(nc));
                    for (uint32_t u = 0; u < nc; ++u) {
                        if (at + u >= sa.chunk_cap) {
                            atomicMax(&M->error, kErrListFull);
                            break;
                        }
                        const uint32_t c0q = lo + u * kSubsetChunk;
                        sa.chunks[at + u] = make_uint4(static_cast<uint32_t>(j), c0q,
                                                       hi - c0q > kSubsetChunk ? c0q + kSubsetChunk : hi,
                                                       piece == 1 ? 1u : 0u);
                    }
                }
                continue;
            }
            for (uint32_t q = lo; q < hi; ++q) {
                if (q == p) continue;
                const bool wm = sa.moved_by_pos[q] != 0;
                const uint32_t idw = (wm || kEmit) ? a.P.id[q] : 0u;
                if (wm && idw < idv) continue;  // a pair of moved vertices once
                if (piece != 1 && !subset_test<kFilter>(a, M, va, vb, p, q, coshR)) continue;
                if (kEmit && out + found < sa.capacity) write_edge<false>(a, out + found, idv, idw);
                ++found;
            }
        }
        if (!kEmit) sa.counts[t] = found;
    }
}

// Chunks of long pieces: one warp per chunk, the candidates over the lanes; the
// chunk's count and pairs use slot count + c of counts / offsets.
template <bool kFilter, bool kEmit>
__global__ void __launch_bounds__(kThreads) subset_chunk_kernel(QueryArgs a, SubsetArgs sa)
{
    Meta *M = a.M;
    if (M->error || (M->filter != 0) != kFilter) return;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const double coshR = M->coshR;
    const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x / 32);
    const uint64_t nch = *sa.chunk_n < sa.chunk_cap ? *sa.chunk_n : sa.chunk_cap;
    for (uint64_t c = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32; c < sa.chunk_cap;
         c += warps) {
        const uint64_t slot = sa.count * M->B + c;
        if (c >= nch) {  // unused slot
            if (!kEmit && lane == 0) sa.counts[slot] = 0;
            continue;
        }
        const uint4 h = sa.chunks[c];  // {owner index, lo, hi, 1 = certain}
        const uint32_t p = sa.owners[h.x];
        const uint32_t idv = a.P.id[p];
        float4 va = make_float4(0, 0, 0, 0), vb = va;
        if (kFilter) {
            const float2 an = a.P.ang[p];
            const float4 q = a.P.pms[p];
            va = make_float4(an.x, an.y, q.x, q.y);
            vb = make_float4(2.0f * q.z, q.x + q.y, kCBase + q.w, 0.0f);
        }
        uint64_t out = 0;
        if (kEmit) out = *sa.base + sa.offsets[slot];
        uint32_t found = 0;
        for (uint32_t q0 = h.y; q0 < h.z; q0 += 32) {
            const uint32_t q = q0 + lane;
            bool edge = false;
            uint32_t idw = 0;
            if (q < h.z && q != p) {
                const bool wm = sa.moved_by_pos[q] != 0;
                if (wm || kEmit) idw = a.P.id[q];
                if (!wm || idv < idw)
                    edge = h.w != 0 || subset_test<kFilter>(a, M, va, vb, p, q, coshR);
            }
            const uint32_t word = __ballot_sync(full, edge);
            if (kEmit && edge) {
                const uint64_t at = out + found + __popc(word & lt);
                if (at < sa.capacity) write_edge<false>(a, at, idv, idw);
            }
            found += __popc(word);
        }
        if (!kEmit && lane == 0) sa.counts[slot] = found;
    }
}

// --------------------------------------------------------------------- CSR finish
// row_ptr[r] = first entry of row r in keys sorted by (row, col); col = low words.
__global__ void csr_finish_kernel(const uint64_t *keys, uint64_t entries, uint64_t n, uint64_t *row_ptr,
                                  uint32_t *col)
{
    for (uint64_t j = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; j < entries;
         j += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t k = keys[j];
        col[j] = static_cast<uint32_t>(k);
        const uint64_t row = k >> 32;
        const uint64_t prev = j ? (keys[j - 1] >> 32) + 1 : 0;  // rows prev..row start at j
        for (uint64_t r = prev; r <= row; ++r) row_ptr[r] = j;
        if (j == entries - 1)
            for (uint64_t r = row + 1; r <= n; ++r) row_ptr[r] = entries;
    }
}

__global__ void fill_u64_kernel(uint64_t *a, uint64_t count, uint64_t v)
{
    for (uint64_t j = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; j < count;
         j += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        a[j] = v;
}

// Bucket index of every band from the sorted keys ((band << 32) | angle key):
// position p writes the entries of the buckets from just after its predecessor's
// bucket up to its own, and the band's last point also the entries after its
// bucket up to the sentinel.
__global__ void __launch_bounds__(kThreads) bucket_index_kernel(const Meta *M, const uint64_t *keys, uint64_t n,
                                                                 uint32_t *idx, uint64_t cap)
{
    if (M->error) return;  // an earlier stage failed: the keys may be undefined
    const uint32_t B = M->B;
    for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t key = keys[p];
        const uint32_t b = static_cast<uint32_t>(key >> 32);
        if (b >= B) {  // cannot happen: every key carries its band
            atomicExch(&const_cast<Meta *>(M)->error, kErrInternal);
            return;
        }
        const uint32_t sh = M->idx_shift[b], off = M->idx_off[b];
        const uint64_t s = M->band_start[b], e = M->band_start[b + 1];
        const uint32_t cur = static_cast<uint32_t>(key) >> sh;
        const uint32_t first = p == s ? 0u : (static_cast<uint32_t>(keys[p - 1]) >> sh) + 1;
        if (off + (1ull << (32 - sh)) >= cap) {  // cannot happen: the offsets are bounded by index_entries(n)
            atomicExch(&const_cast<Meta *>(M)->error, kErrInternal);
            return;
        }
        for (uint32_t j = first; j <= cur; ++j) idx[off + j] = static_cast<uint32_t>(p);
        if (p + 1 == e) {
            const uint32_t nb = 1u << (32 - sh);
            for (uint32_t j = cur + 1; j <= nb; ++j) idx[off + j] = static_cast<uint32_t>(e);
        }
    }
}

// Batch: tile t (one CTA), the tile's graph's bands and index region.
__device__ __forceinline__ void bucket_index_tile(const Meta *metas, const BatchTables &bt, const uint64_t *keys,
                                                  uint32_t *idx, uint32_t t)
{
    const uint4 T = bt.tiles[t];
    const Meta *M = metas + T.x;
    if (M->error || metas[bt.G].error) return;
    const uint32_t B = M->B;
    const uint64_t cap = bt.idx_base[T.x + 1];
    for (uint32_t jj = threadIdx.x; jj < T.z; jj += blockDim.x) {
        const uint64_t p = T.y + jj;
        const uint64_t key = keys[p];
        const uint32_t b = static_cast<uint32_t>(key >> 32);
        if (b >= B) {  // cannot happen: every key carries its band
            atomicExch(const_cast<uint32_t *>(&metas[bt.G].error), kErrInternal);
            return;
        }
        const uint32_t sh = M->idx_shift[b], off = M->idx_off[b];
        const uint64_t s = M->band_start[b], e = M->band_start[b + 1];
        const uint32_t cur = static_cast<uint32_t>(key) >> sh;
        const uint32_t first = p == s ? 0u : (static_cast<uint32_t>(keys[p - 1]) >> sh) + 1;
        if (off + (1ull << (32 - sh)) >= cap) {  // cannot happen: bounded by index_entries(n_g)
            atomicExch(const_cast<uint32_t *>(&metas[bt.G].error), kErrInternal);
            return;
        }
        for (uint32_t j = first; j <= cur; ++j) idx[off + j] = static_cast<uint32_t>(p);
        if (p + 1 == e) {
            const uint32_t nb = 1u << (32 - sh);
            for (uint32_t j = cur + 1; j <= nb; ++j) idx[off + j] = static_cast<uint32_t>(e);
        }
    }
}

// ------------------------------------------------------------ persistent batch
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier of a cooperative launch: every CTA arrives on bar[0]; the last one
// resets it and advances the generation bar[32]; the others wait for the
// generation to change.  A wait gives up after timeout_ns of device time, records
// kErrTimeout in C->error and returns false (so does every CTA that returns
// early: the caller stops).  All threads of the CTA call it.
__device__ bool grid_sync(uint32_t *bar, uint32_t expected, uint64_t timeout_ns, Meta *C)
{
    __shared__ int passed;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t *gen = bar + 32;
        const uint32_t g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) + 1u == expected) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 32, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*gen == g) {
                if (global_ns() - t0 > timeout_ns) {
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        if (!ok) atomicMax(&C->error, kErrTimeout);
        passed = ok;
    }
    __syncthreads();
    return passed != 0;
}

// Shared memory of the persistent kernel: one stage at a time.
union PersistSmem {
    stg::PlanSmem plan;
    stg::SampleSmem sample;
    uint32_t warp_sum[stg::kWarps];
    struct {
        uint32_t off[kMaxBands + 1], bits[kMaxBands];
    } tables;
    struct {
        stg::BucketSmem bucket;
        uint32_t info[kThreads], s[kThreads], cnt[kThreads];
    } slots;
    struct {
        BandShared S[kWarps];
        PerWarp<true, kAccCap> W[kWarps];
    } qf;
    struct {
        BandShared S[kWarps];
        PerWarp<false, kAccCap> W[kWarps];
    } qd;
    WarpSmem heavy[kWarps];
};

constexpr int kPersistMinBlocks = 3;

// The whole batch in one launch (see launch_batch_persistent): stage after stage,
// each spread over all CTAs (tiles and graphs handed out round robin, the range
// query's warp batches from its work counters), separated by grid_sync.
template <bool kVerify>
__global__ void __launch_bounds__(kThreads, kPersistMinBlocks) batch_persistent_kernel(PersistBuffers b, QueryArgs q)
{
    extern __shared__ __align__(16) unsigned char persist_smem[];
    PersistSmem &U = *reinterpret_cast<PersistSmem *>(persist_smem);
    const BatchTables &bt = b.bt;
    const uint32_t G = bt.G, tiles = bt.num_tiles, nblocks = gridDim.x;
    Meta *C = b.metas + G;
    int mark = 0;
    auto sync = [&]() -> bool {
        if (!grid_sync(b.bar, nblocks, b.timeout_ns, C)) return false;
        ++mark;
        if (blockIdx.x == 0 && threadIdx.x == 0 && mark < kMaxStageMarks) C->stage_ns[mark] = global_ns();
        return true;
    };
    const uint64_t t_start = global_ns();
    // plan (one CTA per graph; the last item clears the control block)
    for (uint32_t vb = blockIdx.x; vb <= G; vb += nblocks) stg::plan_batch_item(b.metas, b.args, G, vb, U.plan);
    if (!sync()) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) C->stage_ns[0] = t_start;  // after the plan cleared the block
    for (uint32_t vb = blockIdx.x; vb < tiles; vb += nblocks)
        stg::sample_tile(b.metas, bt, b.keys0, b.r_by_pos, b.bk_counts, vb, U.sample);
    if (!sync()) return;
    // bucket sort (angular sort within each band), the gather fused into its last pass
    for (uint32_t vb = blockIdx.x; vb < G; vb += nblocks)
        stg::bucket_scan_graph(b.metas, bt, b.bk_counts, b.bk_start, b.bk_info, vb, U.warp_sum);
    if (!sync()) return;
    for (uint32_t vb = blockIdx.x; vb < tiles; vb += nblocks)
        stg::bucket_scatter_tile(b.metas, bt, b.keys0, b.bk_counts, b.keys1, vb, U.tables.off, U.tables.bits);
    if (!sync()) return;
    // bucket slots in rounds of kThreads per CTA: each thread looks up one slot, so
    // the unused and empty slots cost no serial loads
    const uint32_t nbk = bt.bk_base[G];
    for (uint32_t r0 = blockIdx.x; r0 < nbk; r0 += kThreads * nblocks) {
        __syncthreads();  // the previous round is done with the slot table
        const uint32_t vb = r0 + threadIdx.x * nblocks;
        uint32_t info = 0xffffffffu, s0 = 0, s1 = 0;
        if (vb < nbk) {
            info = b.bk_info[vb];
            if (info != 0xffffffffu) {
                s0 = b.bk_start[vb];
                s1 = b.bk_start[vb + 1];
            }
        }
        U.slots.info[threadIdx.x] = s1 > s0 ? info : 0xffffffffu;
        U.slots.s[threadIdx.x] = s0;
        U.slots.cnt[threadIdx.x] = s1 - s0;
        __syncthreads();
        for (int t = 0; t < kThreads; ++t) {
            const uint32_t info_t = U.slots.info[t];
            if (info_t == 0xffffffffu) continue;
            stg::bucket_gather_item(b.metas, bt, info_t, U.slots.s[t], U.slots.cnt[t], b.keys1, b.keys0, b.r_by_pos,
                                    b.P, U.slots.bucket);
        }
    }
    if (!sync()) return;
    const uint64_t *kin = b.keys1;
    for (uint32_t vb = blockIdx.x; vb < tiles; vb += nblocks) bucket_index_tile(b.metas, bt, kin, b.bidx, vb);
    if (!sync()) return;
    // range query: the filter graphs, then the FP64 graphs
    batch_body<true, false, true, kVerify>(q, U.qf.S, U.qf.W);
    if (!sync()) return;
    heavy_body<true, false, true, kVerify>(q, U.heavy);
    if (!sync()) return;
    recheck_batch_body(q);
    if (!sync()) return;
    reset_phase(C);
    if (!sync()) return;
    batch_body<false, false, true, kVerify>(q, U.qd.S, U.qd.W);
    if (!sync()) return;
    heavy_body<false, false, true, kVerify>(q, U.heavy);
    if (!sync()) return;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += nblocks * blockDim.x)
        stg::batch_result_one(b.metas, g, b.results);
    if (blockIdx.x == 0 && threadIdx.x == 0 && mark + 1 < kMaxStageMarks) C->stage_ns[mark + 1] = global_ns();
}

__global__ void barrier_test_kernel(Meta *C, uint32_t *bar, uint32_t expected, uint64_t timeout_ns)
{
    grid_sync(bar, expected, timeout_ns, C);
}

template <typename K>
int resident_ctas(K kernel)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
    return (per_sm > 0 ? per_sm : 1) * num_sms();
}

template <bool kFilter, bool kCsr, bool kMulti>
Status run(const QueryArgs &a, cudaStream_t stream)
{
    Status st;
    const uint64_t nbatch = kMulti ? static_cast<uint64_t>(a.bt.num_tiles) * (kTilePoints / 32) : (a.P.n + 31) / 32;
    const uint64_t need = ceil_div(nbatch ? nbatch : 1, kWarps);
    static std::atomic<int> grid_b_cache{0}, grid_h_cache{0};  // filled once; racing threads agree
    int grid_b = grid_b_cache.load(std::memory_order_relaxed), grid_h = grid_h_cache.load(std::memory_order_relaxed);
    if (!grid_b) grid_b_cache.store(grid_b = resident_ctas(batch_kernel<kFilter, kCsr, kMulti, false>),
                                    std::memory_order_relaxed);
    if (!grid_h) grid_h_cache.store(grid_h = resident_ctas(heavy_kernel<kFilter, kCsr, kMulti, false>),
                                    std::memory_order_relaxed);
    const unsigned gb = static_cast<unsigned>(need < static_cast<uint64_t>(grid_b) ? need : grid_b);
    if (a.verify) batch_kernel<kFilter, kCsr, kMulti, true><<<gb, kThreads, 0, stream>>>(a);
    else batch_kernel<kFilter, kCsr, kMulti, false><<<gb, kThreads, 0, stream>>>(a);
    RHG_LAUNCH_CHECK();
    if (a.verify) heavy_kernel<kFilter, kCsr, kMulti, true><<<static_cast<unsigned>(grid_h), kThreads, 0, stream>>>(a);
    else heavy_kernel<kFilter, kCsr, kMulti, false><<<static_cast<unsigned>(grid_h), kThreads, 0, stream>>>(a);
    RHG_LAUNCH_CHECK();
    if (kFilter) {
        recheck_kernel<kCsr><<<static_cast<unsigned>(num_sms() * 4), kThreads, 0, stream>>>(a);
        RHG_LAUNCH_CHECK();
    }
    return st;
}

}  // namespace

Status launch_query(const QueryArgs &a, bool csr, cudaStream_t stream)
{
    Status st;
    if (a.P.n) {
        const uint64_t g = ceil_div(a.P.n, kThreads);
        const uint64_t cap = static_cast<uint64_t>(num_sms()) * 8;
        bucket_index_kernel<<<static_cast<unsigned>(g < cap ? g : cap), kThreads, 0, stream>>>(a.M, a.P.key, a.P.n,
                                                                                                a.bidx, index_entries(a.P.n));
        RHG_LAUNCH_CHECK();
    }
    st = csr ? run<true, true, false>(a, stream) : run<true, false, false>(a, stream);
    if (st.code) return st;
    return csr ? run<false, true, false>(a, stream) : run<false, false, false>(a, stream);
}

Status launch_query_phased(QueryArgs a, uint32_t phases, uint64_t *host_m, cudaEvent_t *events,
                           cudaStream_t stream)
{
    Status st = launch_bucket_index(a, stream);
    if (st.code) return st;
    // phases run from the outermost batches inwards: the first phase, a sixteenth
    // of the batches (rim points, few bands each), ends soon, so the copy of its
    // edges starts early; the rest is split evenly
    const uint64_t nb = (a.P.n + 31) / 32;
    const uint64_t first = phases > 1 ? nb / 16 : nb, rest = nb - first;
    for (uint32_t p = 0; p < phases; ++p) {
        if (p == 0) {
            a.batch_lo = static_cast<uint32_t>(rest);
            a.batch_hi = static_cast<uint32_t>(nb);
        } else {
            a.batch_lo = static_cast<uint32_t>(rest * (phases - 1 - p) / (phases - 1));
            a.batch_hi = static_cast<uint32_t>(rest * (phases - p) / (phases - 1));
        }
        if (a.batch_hi > a.batch_lo) {
            st = run<true, false, false>(a, stream);
            if (st.code) return st;
            st = run<false, false, false>(a, stream);
            if (st.code) return st;
        }
        phase_end_kernel<<<1, 32, 0, stream>>>(a.M, p, a.heavy_cap, a.recheck_cap, host_m);
        RHG_LAUNCH_CHECK();
        if (events) RHG_CUDA_TRY(cudaEventRecord(events[p], stream));
    }
    return st;
}

Status launch_bucket_index(const QueryArgs &a, cudaStream_t stream)
{
    Status st;
    if (a.P.n) {
        const uint64_t g = ceil_div(a.P.n, kThreads);
        const uint64_t cap = static_cast<uint64_t>(num_sms()) * 8;
        bucket_index_kernel<<<static_cast<unsigned>(g < cap ? g : cap), kThreads, 0, stream>>>(a.M, a.P.key, a.P.n,
                                                                                                a.bidx, index_entries(a.P.n));
        RHG_LAUNCH_CHECK();
    }
    return st;
}

Status launch_subset_query(const QueryArgs &a, const uint32_t *owners, uint64_t count,
                           const unsigned long long *owners_found, uint4 *chunks, uint64_t chunk_cap,
                           unsigned long long *chunk_n, const uint8_t *moved_by_pos, uint32_t *counts,
                           const uint64_t *offsets, const unsigned long long *base, uint64_t capacity, bool emit,
                           cudaStream_t stream)
{
    Status st;  // launched even for no moved vertex: the counting pass clears the chunk slots
    const SubsetArgs sa{owners, count, owners_found, chunks, chunk_cap, chunk_n, moved_by_pos, counts, offsets, base,
                        capacity};
    const uint64_t need = ceil_div(count ? count * kMaxBands : 1, kThreads);
    const uint64_t cap = static_cast<uint64_t>(num_sms()) * 16;
    const unsigned g = static_cast<unsigned>(need < cap ? need : cap);
    const unsigned gw = static_cast<unsigned>(num_sms() * 4);
    if (emit) {
        subset_kernel<true, true><<<g, kThreads, 0, stream>>>(a, sa);
        RHG_LAUNCH_CHECK();
        subset_kernel<false, true><<<g, kThreads, 0, stream>>>(a, sa);
        RHG_LAUNCH_CHECK();
        subset_chunk_kernel<true, true><<<gw, kThreads, 0, stream>>>(a, sa);
        RHG_LAUNCH_CHECK();
        subset_chunk_kernel<false, true><<<gw, kThreads, 0, stream>>>(a, sa);
    } else {
        subset_kernel<true, false><<<g, kThreads, 0, stream>>>(a, sa);
        RHG_LAUNCH_CHECK();
        subset_kernel<false, false><<<g, kThreads, 0, stream>>>(a, sa);
        RHG_LAUNCH_CHECK();
        subset_chunk_kernel<true, false><<<gw, kThreads, 0, stream>>>(a, sa);
        RHG_LAUNCH_CHECK();
        subset_chunk_kernel<false, false><<<gw, kThreads, 0, stream>>>(a, sa);
    }
    RHG_LAUNCH_CHECK();
    return st;
}

namespace {

template <bool kVerify>
Status persistent_launch(const PersistBuffers &b, cudaStream_t stream)
{
    Status st;
    auto kernel = batch_persistent_kernel<kVerify>;
    const int smem = static_cast<int>(sizeof(PersistSmem));
    static std::atomic<int> grid_cache{0};  // filled once; racing threads agree
    int grid = grid_cache.load(std::memory_order_relaxed);
    if (!grid) {
        RHG_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int per_sm = 0;
        RHG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem));
        grid = (per_sm > 0 ? per_sm : 1) * num_sms();
        grid_cache.store(grid, std::memory_order_relaxed);
    }
    QueryArgs q{};
    q.M = b.metas;
    q.bt = b.bt;
    q.P = b.P;
    q.pairs = b.pairs;
    q.heavy = b.heavy;
    q.heavy_cap = b.heavy_cap;
    q.recheck = b.recheck;
    q.recheck_cap = b.recheck_cap;
    q.bidx = b.bidx;
    q.verify = kVerify;
    void *args[] = {const_cast<PersistBuffers *>(&b), &q};
    RHG_CUDA_TRY(cudaMemsetAsync(b.bar, 0, 256, stream));
    RHG_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kernel), dim3(grid), dim3(kThreads), args,
                                             smem, stream));
    RHG_LAUNCH_CHECK();
    return st;
}

}  // namespace

Status launch_batch_persistent(const PersistBuffers &b, bool verify, cudaStream_t stream)
{
    if (b.bt.num_tiles == 0 || b.bt.G == 0) return Status{};
    return verify ? persistent_launch<true>(b, stream) : persistent_launch<false>(b, stream);
}

Status launch_barrier_test(Meta *C, uint32_t *bar, uint32_t missing, uint64_t timeout_ns, cudaStream_t stream)
{
    Status st;
    const int grid = 2 * num_sms();  // two CTAs of 32 threads per SM are always co-resident
    const uint32_t expected = static_cast<uint32_t>(grid) + missing;
    void *args[] = {&C, &bar, const_cast<uint32_t *>(&expected), &timeout_ns};
    RHG_CUDA_TRY(cudaMemsetAsync(bar, 0, 256, stream));
    RHG_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(barrier_test_kernel), dim3(grid), dim3(32),
                                             args, 0, stream));
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_csr_finish(const uint64_t *sorted_keys, uint64_t entries, uint64_t n, uint64_t *row_ptr,
                         uint32_t *col, cudaStream_t stream)
{
    Status st;
    if (entries == 0) {
        const uint64_t g = ceil_div(n + 1, 256);
        fill_u64_kernel<<<static_cast<unsigned>(g < 4096 ? g : 4096), 256, 0, stream>>>(row_ptr, n + 1, 0);
    } else {
        const uint64_t need = ceil_div(entries, 256);
        const uint64_t cap = static_cast<uint64_t>(num_sms()) * 16;
        csr_finish_kernel<<<static_cast<unsigned>(need < cap ? need : cap), 256, 0, stream>>>(
            sorted_keys, entries, n, row_ptr, col);
    }
    RHG_LAUNCH_CHECK();
    return st;
}

}  // namespace rhg
