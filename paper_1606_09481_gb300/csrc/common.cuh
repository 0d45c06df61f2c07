// common.cuh -- shared definitions of the CUDA path: per-graph metadata kept in
// device memory, the counter-based generator, the canonical edge predicate and
// error-checking helpers.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include <cstdint>

#include "../../include/rhg.h"
#include "detmath.cuh"

namespace rhg {

constexpr int kMaxBands = static_cast<int>(RHG_MAX_BANDS);
// bucket index: about kBucketPoints..2 kBucketPoints points per bucket, at least
// two buckets per band; index_entries(n) bounds the entries of all bands
constexpr uint32_t kBucketPoints = 1;
__host__ __device__ constexpr uint64_t index_entries(uint64_t n) { return n / kBucketPoints + 3 * kMaxBands + 1; }
constexpr int kExpTab = 64;  // e^k table for k = -64..64 (FP32 filter values)
constexpr int kYTab = 66;    // 2^(+-e/alpha) e^-G tables for the exponents e = 0..65 of y (filter_values_u53)
constexpr uint32_t kClaimCounters = 16;  // work-claim counters of the range query (Meta::claim)
// bucket sort of generated points (angular sort within each band): band j is cut
// into 2^bits_j buckets by the top bits of the angle key, about kBucketTarget to
// 2 kBucketTarget expected points each; buckets of up to kBucketCap points are
// sorted in shared memory.  bucket_entries(n) bounds the buckets of all bands.
constexpr uint32_t kBucketTarget = 512;
constexpr uint32_t kBucketCap = 2048;
__host__ __device__ constexpr uint64_t bucket_entries(uint64_t n) { return n / kBucketTarget + kMaxBands + 1; }
constexpr int kMaxStageMarks = 32;       // stage timestamps of the persistent batch launch
constexpr int kMaxPhases = 16;           // phases of a range query whose output is copied out as it goes

// ---------------------------------------------------------------------------
// FP32 filter: error model.  The filter evaluates X = L / cosh R in the
// cancellation-free form X = P_v M_w + M_v P_w + 2 S_v S_w sin^2(d/2) with
// P = e^{r - G}, M = e^{-r - G}, S = sinh(r) e^{-G} sqrt 2, G = ln(2 cosh R)/2,
// all FP32, and decides only when |X - 1| exceeds a bound on every error
// between X and the rounded FP64 predicate (Eq. 3); other pairs are rechecked
// with the FP64 predicate itself.
constexpr double kDeltaR = 1e-6;        // slack on the band radii of the FP32 windows (band members
                                         // are within 1e-13 of their band: see band_of_u53)
constexpr float kEpsPM = 2e-6f;          // relative error of stored P and M (analysis: <= 1.2e-6,
                                         // filter_values_u53; <= 8.4e-7 from an FP64 radius)
constexpr float kEps32 = 5.9604645e-8f;  // 2^-24
constexpr float kCBase = 6e-6f;          // 2 kEpsPM + 8 eps32 + 2 eps_sin, rounded up
constexpr float kAngAbs = 2e-13f;        // absolute error of |phi_v - phi_w| from the hi/lo split, x2
constexpr float kC64 = 3.56e-15f;        // 32 u (1 + 1e-3): |L - X H| / H <= kC64 (P_v+M_v)(P_w+M_w)
constexpr double kFilterMaxR = 32.0;     // above this the FP64 noise of Eq. 3 makes the filter useless
constexpr double kFilterMaxAlphaR = 44.0;  // w (w + 2) finite in FP32: w <= cosh(alpha R) - 1 < 1.84e19

// Per-graph metadata, written by the plan kernel and read by all later stages.
struct Meta {
    double R;          // disk radius
    double coshR;      // dm::cosh(R): the predicate's threshold
    double alpha;
    double inv_alpha;  // 1 / alpha
    double cm1;        // dm::cosh(alpha R) - 1 (inverse CDF of Eq. 1)
    double G;          // ln(2 cosh R) / 2 (FP32 filter scaling)
    double c[kMaxBands + 1];        // band boundaries c_0 = 0 .. c_B = R
    double cosh_c[kMaxBands + 1];   // cosh / sinh of the boundaries (FP64 windows)
    double sinh_c[kMaxBands + 1];
    uint64_t band_start[kMaxBands + 1];  // sorted position of each band's first point
    uint32_t band_count[kMaxBands];
    // bucket index of band i (range query search): entries idx_off[i] ..
    // idx_off[i] + 2^(32 - idx_shift[i]); entry j = first position of the band
    // whose angle key >> idx_shift[i] is >= j
    uint32_t idx_off[kMaxBands + 1];
    uint32_t idx_shift[kMaxBands];
    // FP32 window constants of band i: inner radius c_i - kDeltaR, outer c_{i+1} + kDeltaR
    float band_P[kMaxBands + 1], band_M[kMaxBands + 1], band_S[kMaxBands + 1];
    float band_PMn[kMaxBands + 1];  // P + M at the outer radius
    float band_Po[kMaxBands + 1], band_Mo[kMaxBands + 1], band_So[kMaxBands + 1];  // at the outer radius
    float etab[2 * kExpTab + 1];    // e^k rounded to float
    // generated points in filter mode (band_of_u53, filter_values_u53): band j holds
    // the radial variates band_u[j] <= u53 < band_u[j + 1]; y = 2^e m gives
    // P = tabP[e] m^(1/alpha), M = tabM[e] m^(-1/alpha)
    uint64_t band_u[kMaxBands + 1];
    float tabP[kYTab], tabM[kYTab];  // 2^(e/alpha) e^-G, 2^(-e/alpha) e^-G rounded to float
    float cw;                        // (cosh(alpha R) - 1) 2^-53 rounded to float
    float inv_alpha_f;               // 1 / alpha rounded to float
    float y_one;                     // e^alpha rounded to float: y >= y_one means r >= 1 (about)
    uint32_t alpha_one;              // alpha == 1: m^(1/alpha) = m exactly
    // buckets of the sort (generated points): band j holds the buckets
    // bk_off[j] .. bk_off[j+1]-1, bucket = bk_off[j] + (angle key >> (32 - bk_bits[j]))
    uint32_t bk_off[kMaxBands + 1];
    uint32_t bk_bits[kMaxBands];
    uint32_t nbuckets;
    uint32_t B;
    uint32_t batch_budget, core_heavy, fringe_limit;  // work mapping of the range query
    uint32_t error;          // nonzero: a device-side check failed (see kErr*)
    uint32_t filter;         // 1: FP32 filter + FP64 recheck; 0: FP64 predicate per candidate
    uint32_t verify;         // 1: check every filter decision against the FP64 predicate
    uint64_t n;
    uint64_t seed;
    double k;
    uint64_t m;              // edges found (exact), also the output cursor
    uint64_t candidates;
    uint64_t near_threshold;  // FP64-decided pairs with |L - cosh R| <= 1e-12 cosh R
    uint64_t rounding_band;   // FP64-decided pairs with |L - cosh R| <= 8 u cosh r_v cosh r_w
    uint64_t rechecks;
    uint64_t verify_failures;
    uint32_t heavy_n, heavy_next;      // heavy-range chunk list
    uint32_t recheck_n, pad0;          // FP64 recheck list
    uint32_t heavy_lo, recheck_lo;     // phased query: entries before these are done
    uint64_t m_phase[kMaxPhases];      // phased query: the edge count after each phase
    uint64_t work_counter;             // dynamic model: moved vertices listed
    // work claims of the range query: counter c hands out the warp batches
    // c, c + kClaimCounters, ... (one counter per 128-byte line, so that the claims
    // of different warps do not queue on one address)
    uint32_t claim[kClaimCounters * 32];
    // persistent batch launch (control block): the device time (globaltimer, ns)
    // at the start and after each stage's grid barrier
    uint64_t stage_ns[kMaxStageMarks];
};

// device-side error codes (Meta::error)
constexpr uint32_t kErrNone = 0;
constexpr uint32_t kErrNoSolution = 1;
constexpr uint32_t kErrBadPoint = 2;
constexpr uint32_t kErrTimeout = 3;
constexpr uint32_t kErrInternal = 4;
constexpr uint32_t kErrListFull = 5;  // heavy or recheck list overflowed: rerun in FP64 mode

// ----------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 64x64->128
// multiplications with the published multipliers, key schedule by the published
// Weyl increments.
struct U64x4 {
    uint64_t x0, x1, x2, x3;
};

__device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, uint64_t k0, uint64_t k1)
{
    constexpr uint64_t kMul0 = 0xD2E7470EE14C6C93ULL, kMul1 = 0xCA5A826395121157ULL;
    constexpr uint64_t kWeyl0 = 0x9E3779B97F4A7C15ULL, kWeyl1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += kWeyl0;
            k1 += kWeyl1;
        }
        const uint64_t hi0 = __umul64hi(kMul0, c.x0), lo0 = kMul0 * c.x0;
        const uint64_t hi1 = __umul64hi(kMul1, c.x2), lo1 = kMul1 * c.x2;
        c = U64x4{hi1 ^ c.x1 ^ k0, lo1, hi0 ^ c.x3 ^ k1, lo0};
    }
    return c;
}

// Angle of point `id`: phi = fl(u53 * 2pi 2^-53), u53 = top 53 bits of word 0.
constexpr double kPhiScale = 0x1.921fb54442d18p-51;  // kTwoPi * 2^-53, exact
constexpr double kU53 = 0x1.0p-53;

// Search key of an angle: floor(phi * 2^32 / 2pi) clamped to [0, 2^32 - 1]; a
// monotone map of phi, so that key order refines angle order.
constexpr double kKeyScale = 0x1.45f306dc9c883p+29;  // nearest double to 2^32 / (2 pi)

__device__ __forceinline__ uint32_t angle_key(double phi)
{
    const double t = floor(__dmul_rn(phi, kKeyScale));
    if (!(t > 0.0)) return 0u;
    if (t >= 4294967295.0) return 0xffffffffu;
    return static_cast<uint32_t>(t);
}

// Radial coordinate from its uniform variate (inverse CDF of Eq. 1):
//   w = U (cosh(alpha R) - 1),  r = ln(1 + w + sqrt(w (w + 2))) / alpha, clamped to R.
__device__ __forceinline__ double radius_from_u53(uint64_t u53, double R, double cm1,
                                                  double inv_alpha)
{
    const double U = __dmul_rn(static_cast<double>(u53), kU53);
    const double w = __dmul_rn(U, cm1);
    const double sq = __dsqrt_rn(__dmul_rn(w, __dadd_rn(w, 2.0)));
    const double y = __dadd_rn(__dadd_rn(1.0, w), sq);
    const double r = __dmul_rn(dm::log(y), inv_alpha);
    return r > R ? R : r;
}

__device__ __forceinline__ double phi_from_u53(uint64_t u53)
{
    const double ph = __dmul_rn(static_cast<double>(u53), kPhiScale);
    return ph < dm::kTwoPi ? ph : 0x1.921fb54442d17p+2;  // largest double below 2pi
}

// Philox block of point `id`: word 0 -> angle, word 1 -> radius.
__device__ __forceinline__ U64x4 draw(uint64_t id, uint64_t seed)
{
    return philox4x64_10(U64x4{id, 0, 0, 0}, seed, 0);
}

// ---------------------------------------------------------------------------
// Generated points in filter mode: band and filter values without FP64 (GB300's
// FP64 pipe runs at a small fraction of its integer and FP32 pipes).

// 2^e as a float, e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Band of a generated point from its radial variate u53: the largest j < B with
// bu[j] <= u53, where bu[j] = ceil(F(c_j) 2^53) and F(c) = (cosh(alpha c) - 1) /
// (cosh(alpha R) - 1) is the CDF of Eq. 1 (bu[0] = 0, bu[B] = 2^53).  A variate at
// or above bu[j] has U >= F(c_j) (1 - 1e-15), so its FP64 radius (radius_from_u53)
// is at least c_j - 1e-13; below bu[j + 1] it is at most c_{j+1} + 1e-13.  Integer
// compares only: the FP64 radius is never formed.
__device__ __forceinline__ uint32_t band_of_u53(uint64_t u53, const uint64_t *bu, uint32_t B)
{
    uint32_t lo = 0, hi = B;  // invariant: bu[lo] <= u53, answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (bu[mid] <= u53) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Sort bucket of key = (band << 32) | angle key (band < B; see Meta::bk_off).
__device__ __forceinline__ uint32_t bucket_of(uint64_t key, const uint32_t *off, const uint32_t *bits)
{
    const uint32_t b = static_cast<uint32_t>(key >> 32), nb = bits[b];
    return off[b] + (nb ? static_cast<uint32_t>(key) >> (32 - nb) : 0u);
}

// The angle's hi/lo float pair float(phi), float(phi - float(phi)) for phi =
// fl(u53 kPhiScale) (phi_from_u53, including its clamp below 2 pi), bit for bit,
// with integer arithmetic: kPhiScale = kSig 2^-103 with the 53-bit significand kSig
// of 2 pi, so phi is the 106-bit product u53 kSig rounded to 53 bits (to nearest,
// ties to even, as the FP64 multiplication rounds); hi is that rounded to 24 bits
// the same way, and phi - hi (exact in 30 bits) is rounded to float by the
// integer-to-float conversion.
__device__ __forceinline__ float2 angle_hilo_u53(uint64_t u)
{
    constexpr uint64_t kSig = 0x1921fb54442d18ull;
    if (u == 0) return make_float2(0.0f, 0.0f);
    const uint64_t plo = u * kSig, phi = __umul64hi(u, kSig);
    const int nb = phi ? 128 - __clzll(static_cast<long long>(phi)) : 64 - __clzll(static_cast<long long>(plo));
    int sh = nb - 53;  // 0..53: the product >> sh has 53 bits (kSig has 53, u >= 1)
    uint64_t q = sh ? (plo >> sh) | (phi << (64 - sh)) : plo;
    if (sh) {
        const uint64_t rem = plo & ((uint64_t{1} << sh) - 1), half = uint64_t{1} << (sh - 1);
        if (rem > half || (rem == half && (q & 1u))) {
            if (++q == (uint64_t{1} << 53)) {
                q >>= 1;
                ++sh;
            }
        }
    }
    // phi = q 2^(sh - 103); 2 pi = kSig 2^-50
    if (sh > 53 || (sh == 53 && q >= kSig)) {
        q = kSig - 1;  // the largest double below 2 pi
        sh = 53;
    }
    uint64_t h = q >> 29;
    const uint64_t r = q & 0x1fffffffull;
    if (r > 0x10000000ull || (r == 0x10000000ull && (h & 1u))) ++h;  // h <= 2^24
    const int lo_i = static_cast<int>(static_cast<int64_t>(q) - static_cast<int64_t>(h << 29));  // |.| <= 2^28
    return make_float2(__uint2float_rn(static_cast<uint32_t>(h)) * pow2f(sh - 74),
                       __int2float_rn(lo_i) * pow2f(sh - 103));
}

// u53 rounded to float (to nearest, ties to even), with integer arithmetic.
__device__ __forceinline__ float u53_to_float(uint64_t u)
{
    if (u < (uint64_t{1} << 24)) return __uint2float_rn(static_cast<uint32_t>(u));
    const int s = 40 - __clzll(static_cast<long long>(u));  // bit length - 24, 1..29
    uint64_t m = u >> s;
    const uint64_t rem = u & ((uint64_t{1} << s) - 1), half = uint64_t{1} << (s - 1);
    if (rem > half || (rem == half && (m & 1u))) ++m;  // m <= 2^24
    return __uint2float_rn(static_cast<uint32_t>(m)) * pow2f(s);
}

// The sampler's FP64 angle and radius of point `id` (Alg. 1, Eq. 1).
__device__ __forceinline__ void point_fp64(uint64_t id, uint64_t seed, double R, double cm1, double inv_alpha,
                                           double *ph, double *r)
{
    const U64x4 x = draw(id, seed);
    *ph = phi_from_u53(x.x0 >> 11);
    *r = radius_from_u53(x.x1 >> 11, R, cm1, inv_alpha);
}

// Canonical edge predicate (Eq. 3, threshold test of Alg. 1): returns L; the
// pair is an edge iff L <= cosh R.
__device__ __forceinline__ double predicate_L(double phv, double chv, double shv, double phw,
                                              double chw, double shw)
{
    const double d = fabs(__dsub_rn(phv, phw));
    const double c = dm::cos(d);
    const double t1 = __dmul_rn(chv, chw);
    const double t3 = __dmul_rn(__dmul_rn(shv, shw), c);
    return __dsub_rn(t1, t3);
}

// Band of r: the largest j < B with c_j <= r (Sec. III-A: c_j <= r < c_{j+1}).
__device__ __forceinline__ uint32_t band_of(double r, const double *c, uint32_t B)
{
    uint32_t lo = 0, hi = B;  // invariant: c[lo] <= r, answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (c[mid] <= r) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ----------------------------------------------------------------------------
// host-side helpers
struct Status {
    int code = RHG_OK;
    cudaError_t cuda = cudaSuccess;
};

#define RHG_CUDA_TRY(expr)                                \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) {                          \
            st.code = RHG_ERR_CUDA;                       \
            st.cuda = _e;                                 \
            return st;                                    \
        }                                                 \
    } while (0)

// Kernels launched by the library (rhg_launch_count); every launch site is
// followed by RHG_LAUNCH_CHECK, which counts it.
void note_launch();

#define RHG_LAUNCH_CHECK()                                \
    do {                                                  \
        ::rhg::note_launch();                             \
        cudaError_t _e = cudaGetLastError();              \
        if (_e != cudaSuccess) {                          \
            st.code = RHG_ERR_CUDA;                       \
            st.cuda = _e;                                 \
            return st;                                    \
        }                                                 \
    } while (0)

inline int num_sms()
{
    static std::atomic<int> cached{0};  // host threads may race to fill it; all write the same value
    int sms = cached.load(std::memory_order_relaxed);
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        cached.store(sms, std::memory_order_relaxed);
    }
    return sms;
}

inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

}  // namespace rhg
