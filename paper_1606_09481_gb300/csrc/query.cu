// query.cu -- the range query of Alg. 1, the loop that dominates the running time
// (Sec. III-B): for each point v and each band b_i from v's own band outward, the
// getMinMaxPhi window, a binary search for the first and last candidate in the
// band's angle-sorted keys, and the distance test of every candidate (Eq. 3).
//
// Work decomposition (GB300): a warp takes a batch of 32 consecutive sorted points
// (lane = point) and walks the bands; each lane computes its window and key range,
// and the non-empty (owner, range) entries are queued in shared memory.  A flush
// then lets all 32 lanes test one owner's candidates at a time, writing one
// decision bit per candidate, reserves the batch's output with one atomic add and
// replays the bits to write the pairs.  Ranges longer than kHeavy candidates are
// cut into chunks that a second kernel spreads over all warps (hub vertices).
//
// Candidate test: in filter mode an FP32 test of X = L / cosh R written without
// cancellation, X = P_v M_w + M_v P_w + 2 S_v S_w sin^2(d/2), that decides only when
// |X - 1| exceeds a bound on all errors, including the rounding of the FP64
// predicate itself; undecided pairs are queued and the third kernel evaluates the
// FP64 predicate on them.  FP64 mode evaluates the FP64 predicate directly.
#include "kernels.h"

namespace rhg {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kChunk = 4096;  // candidates per heavy chunk
constexpr int kListCap = 64;       // queued (owner, range) entries per warp (>= 2 per lane)
constexpr int kBitWords = 128;     // decision words per warp: kChunk / 32
constexpr uint32_t kFull = 0x80000000u;  // window half-width meaning "whole band"

constexpr float kPiF = 3.14159265f;             // below pi: the unwrapped branch is safe to pi
constexpr float kTwoPiHiF = 6.28318548202514648f;
constexpr float kTwoPiLoF = -1.74845553e-07f;    // 2 pi - kTwoPiHiF
constexpr float kKeyPerRadF = 683565248.0f;      // 2^32 / (2 pi) in FP32
constexpr double kKeyPerRad = 683565275.57643158;
constexpr float kWinE1 = 5e-6f;                  // window numerator error, relative to 1 + T

struct BandShared {
    uint32_t start[kMaxBands + 1];
    float P[kMaxBands + 1], Mm[kMaxBands + 1], S[kMaxBands + 1], PMn[kMaxBands + 1];
    double c[kMaxBands + 1], sinh_c[kMaxBands + 1], cosh_c[kMaxBands + 1];
};

__device__ __forceinline__ void load_bands(BandShared &S, const Meta *M)
{
    for (int j = threadIdx.x; j <= kMaxBands; j += blockDim.x) {
        S.start[j] = static_cast<uint32_t>(M->band_start[j]);
        S.P[j] = M->band_P[j];
        S.Mm[j] = M->band_M[j];
        S.S[j] = M->band_S[j];
        S.PMn[j] = M->band_PMn[j];
        S.c[j] = M->c[j];
        S.sinh_c[j] = M->sinh_c[j];
        S.cosh_c[j] = M->cosh_c[j];
    }
}

// The owner of a range: the point whose neighbours are searched.
struct Owner {
    uint32_t p, id;
    // filter mode
    float ah, al, P, M, S2, PM, crel, gam;
    // FP64 mode
    double phi, r, ch, sh;
};

template <bool kFilter>
__device__ __forceinline__ Owner load_owner(const SortedPoints &P, uint32_t p)
{
    Owner o;
    o.p = p;
    o.id = P.id[p];
    if (kFilter) {
        const float2 a = P.ang[p];
        const float4 q = P.pms[p];
        o.ah = a.x;
        o.al = a.y;
        o.P = q.x;
        o.M = q.y;
        o.S2 = 2.0f * q.z;
        o.PM = q.x + q.y;
        o.gam = q.w;
        o.crel = kCBase + q.w;
    } else {
        o.phi = P.phi[p];
        o.r = P.r[p];
        o.ch = P.ch[p];
        o.sh = P.sh[p];
    }
    return o;
}

template <bool kFilter>
__device__ __forceinline__ Owner shfl_owner(const Owner &v, int src)
{
    Owner o;
    const unsigned full = 0xffffffffu;
    o.p = __shfl_sync(full, v.p, src);
    o.id = __shfl_sync(full, v.id, src);
    if (kFilter) {
        o.ah = __shfl_sync(full, v.ah, src);
        o.al = __shfl_sync(full, v.al, src);
        o.P = __shfl_sync(full, v.P, src);
        o.M = __shfl_sync(full, v.M, src);
        o.S2 = __shfl_sync(full, v.S2, src);
        o.PM = __shfl_sync(full, v.PM, src);
        o.crel = __shfl_sync(full, v.crel, src);
    } else {
        o.phi = __shfl_sync(full, v.phi, src);
        o.ch = __shfl_sync(full, v.ch, src);
        o.sh = __shfl_sync(full, v.sh, src);
    }
    return o;
}

// FP32 filter: 1 = edge, 0 = no edge, 2 = undecided (FP64 recheck).
//   d    circular |phi_v - phi_w| from hi/lo floats (relative error ~2^-23 plus an
//        absolute error < kAngAbs / 2 from the hi/lo representation)
//   t    sin(d/2), odd Taylor polynomial to x^11 on [0, pi/2] (rel. error ~3 ulp)
//   X    P_v M_w + M_v P_w + 2 S_v S_w t^2
//   err  X (kCBase + gamma_v + gamma_w + kAngAbs / d) + kC64 (P_v + M_v)(P_w + M_w)
__device__ __forceinline__ int filter_decide(const Owner &v, float2 aw, float4 w)
{
    const float dh = v.ah - aw.x;  // correctly rounded: relative error <= 2^-24
    float d;
    if (fabsf(dh) > kPiF) {
        // across 0 / 2 pi: 2 pi - (big - small) = (2 pi_hi - big_hi) + small_hi + lo parts;
        // 2 pi_hi - big_hi is exact (Sterbenz, big > pi), so no absolute error of
        // order ulp(2 pi) enters the small result
        const bool vbig = dh > 0.0f;
        const float bh = vbig ? v.ah : aw.x, bl = vbig ? v.al : aw.y;
        const float sh = vbig ? aw.x : v.ah, sl = vbig ? aw.y : v.al;
        d = ((kTwoPiHiF - bh) + sh) + ((kTwoPiLoF - bl) + sl);
    } else {
        d = fabsf(dh + (v.al - aw.y));
    }
    const float x = 0.5f * d;
    const float z = x * x;
    float t = fmaf(z, -2.50521079e-08f, 2.75573188e-06f);
    t = fmaf(z, t, -1.98412701e-04f);
    t = fmaf(z, t, 8.33333377e-03f);
    t = fmaf(z, t, -1.66666672e-01f);
    t = fmaf(z * x, t, x);
    const float X = fmaf(v.S2 * w.z, t * t, fmaf(v.P, w.y, v.M * w.x));
    const float Q = v.PM * (w.x + w.y);
    const float rel = v.crel + w.w + __fdividef(kAngAbs, d);
    const float err = fmaf(X, rel, kC64 * Q);
    if (X + err <= 1.0f) return 1;
    if (X - err > 1.0f) return 0;
    return 2;
}

// Window half-width in angle-key units (kFull: the whole band).  Filter mode,
// for band i with inner radius c' = c_i - kDeltaR: sin^2(theta/2) =
// (beta - cosh(r_v - c')/cosh R) / (2 sinh r_v sinh c' / cosh R), beta = 1 + the
// FP64 predicate's error bound for r_w < c_{i+1} + kDeltaR, all from the stored
// P, M, S with their error bounds added.
__device__ __forceinline__ uint32_t window_filter(const Owner &v, const BandShared &S, uint32_t i)
{
    const float Sc = S.S[i];
    if (i == 0 || !(Sc > 0.0f) || !(v.S2 > 0.0f)) return kFull;
    const float T = fmaf(v.P, S.Mm[i], v.M * S.P[i]);
    const float beta = fmaf(kC64 * v.PM, S.PMn[i], 1.0f);
    const float num = fmaf(1.0f + T, kWinE1, beta - T);
    const float den = v.S2 * Sc * (1.0f - (v.gam + 6.0f * kEps32));
    const float Q = num / den;
    if (!(Q < 1.0f)) return kFull;
    const float th = 2.0f * asinf(sqrtf(fmaxf(Q, 0.0f)));
    const float keys = fmaf(th, kKeyPerRadF * (1.0f + 2e-5f), 3.0f);
    return keys >= 2147483648.0f ? kFull : static_cast<uint32_t>(keys);
}

// FP64 mode window from the FP64 radius (Sec. III-B getMinMaxPhi), conservative
// for the rounded predicate: threshold (cosh R + 64 u cosh r_v cosh c_{i+1})(1 + 1e-12).
__device__ __forceinline__ uint32_t window_fp64(const Owner &v, const BandShared &S, uint32_t i, double coshR)
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

__device__ __forceinline__ void push_heavy(const QueryArgs &a, uint32_t p, uint32_t lo, uint32_t hi)
{
    const uint32_t nch = (hi - lo + kChunk - 1) / kChunk;
    const uint32_t at = atomicAdd(&a.M->heavy_n, nch);
    if (at + nch > a.heavy_cap || at + nch < at) {
        atomicMax(&a.M->error, kErrListFull);
        return;
    }
    for (uint32_t j = 0; j < nch; ++j) {
        const uint32_t c0 = lo + j * kChunk;
        const uint32_t c1 = hi - c0 > kChunk ? c0 + kChunk : hi;
        a.heavy[at + j] = make_uint4(p, c0, c1, 0u);
    }
}

template <bool kCsr>
__device__ __forceinline__ void write_edge(const QueryArgs &a, uint64_t pos, uint32_t i1, uint32_t i2)
{
    const uint32_t u = i1 < i2 ? i1 : i2, v = i1 < i2 ? i2 : i1;
    if (kCsr) {
        a.csr_keys[2 * pos] = (static_cast<uint64_t>(u) << 32) | v;
        a.csr_keys[2 * pos + 1] = (static_cast<uint64_t>(v) << 32) | u;
    } else {
        reinterpret_cast<uint2 *>(a.pairs)[pos] = make_uint2(u, v);
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

// Verification mode: the FP64 predicate for a pair the filter decided; a
// contradiction, or a decided pair within 1e-12 of the threshold, is counted.
__device__ __noinline__ void verify_pair(const QueryArgs &a, uint32_t idv, uint32_t idw, int dec, double coshR)
{
    double pv, cv, sv, pw, cw, sw;
    fp64_point(a, a.M, idv, pv, cv, sv);
    fp64_point(a, a.M, idw, pw, cw, sw);
    const double L = predicate_L(pv, cv, sv, pw, cw, sw);
    if ((L <= coshR) != (dec == 1) || fabs(L - coshR) <= 1e-12 * coshR)
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.M->verify_failures), 1ull);
}

// Decide candidate q for owner v; queue undecided pairs; in verification mode
// compare every decided pair with the FP64 predicate.
template <bool kFilter>
__device__ __forceinline__ int decide(const QueryArgs &a, const Owner &v, uint32_t q, bool in, double coshR,
                                      bool verify, uint32_t &near)
{
    const unsigned full = 0xffffffffu;
    int dec = 0;
    if (kFilter) {
        if (in) dec = filter_decide(v, a.P.ang[q], a.P.pms[q]);
        const uint32_t um = __ballot_sync(full, dec == 2);
        if (um) {
            const int lane = threadIdx.x & 31;
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&a.M->recheck_n, static_cast<uint32_t>(__popc(um)));
            base = __shfl_sync(full, base, 0);
            if (dec == 2) {
                const uint32_t at = base + __popc(um & ((1u << lane) - 1u));
                if (at < a.recheck_cap) a.recheck[at] = make_uint2(v.p, q);
                else atomicMax(&a.M->error, kErrListFull);
            }
        }
        if (verify && in && dec != 2) verify_pair(a, v.id, a.P.id[q], dec, coshR);
    } else if (in) {
        const double L = predicate_L(v.phi, v.ch, v.sh, a.P.phi[q], a.P.ch[q], a.P.sh[q]);
        dec = L <= coshR;
        near += fabs(L - coshR) <= 1e-12 * coshR;
    }
    return dec;
}

struct WarpSmem {
    uint32_t lo[kListCap], hi[kListCap];
    uint32_t own[kListCap];
    uint32_t bits[kBitWords];
};

// Decide, reserve and write the queued entries [0, count) of this warp, in
// segments of at most kBitWords decision words; an entry longer than a segment
// is continued in the next one.
template <bool kFilter, bool kCsr>
__device__ __forceinline__ void flush(const QueryArgs &a, WarpSmem &W, int count, const Owner &mine, double coshR,
                                      bool verify, uint32_t &near)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    int e = 0;
    uint32_t qpos = count ? W.lo[0] : 0;  // next candidate of entry e
    while (e < count) {
        const int e_start = e;
        const uint32_t q_start = qpos;
        int words = 0;
        uint32_t edges = 0;
        while (e < count && words < kBitWords) {
            const uint32_t hi = W.hi[e];
            const Owner v = shfl_owner<kFilter>(mine, static_cast<int>(W.own[e]));
            for (; qpos < hi && words < kBitWords; qpos += 32) {
                const uint32_t q = qpos + lane;
                const int dec = decide<kFilter>(a, v, q, q < hi, coshR, verify, near);
                const uint32_t word = __ballot_sync(full, dec == 1);
                if (lane == 0) W.bits[words] = word;
                ++words;
                edges += __popc(word);
            }
            if (qpos >= hi) {
                ++e;
                if (e < count) qpos = W.lo[e];
            }
        }
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0 && edges) base = atomicAdd(reinterpret_cast<unsigned long long *>(&a.M->m), edges);
        base = __shfl_sync(full, base, 0);
        if (edges && base + edges <= a.capacity) {
            int wi = 0, ee = e_start;
            uint32_t qq = q_start, run = 0;
            while (wi < words) {
                const uint32_t hi = W.hi[ee];
                const uint32_t idv = __shfl_sync(full, mine.id, static_cast<int>(W.own[ee]));
                for (; qq < hi && wi < words; qq += 32) {
                    const uint32_t word = W.bits[wi++];
                    if ((word >> lane) & 1u) write_edge<kCsr>(a, base + run + __popc(word & lt), idv, a.P.id[qq + lane]);
                    run += __popc(word);
                }
                if (qq >= hi) {
                    ++ee;
                    if (ee < count) qq = W.lo[ee];
                }
            }
        }
        __syncwarp();
    }
}

template <bool kFilter, bool kCsr>
__global__ void __launch_bounds__(kThreads) batch_kernel(QueryArgs a)
{
    __shared__ BandShared S;
    __shared__ WarpSmem Wsm[kWarps];
    Meta *M = a.M;
    load_bands(S, M);
    __syncthreads();
    if (M->error || (M->filter != 0) != kFilter) return;
    const unsigned full = 0xffffffffu;
    const uint32_t n = static_cast<uint32_t>(a.P.n), B = M->B;
    const double coshR = M->coshR;
    const bool verify = M->verify != 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem &W = Wsm[warp];
    const uint32_t nbatch = (n + 31) / 32;
    unsigned long long cand = 0;
    uint32_t near = 0;
    for (uint32_t batch = blockIdx.x * kWarps + warp; batch < nbatch; batch += gridDim.x * kWarps) {
        const uint32_t p = batch * 32 + lane;
        const bool valid = p < n;
        Owner mine{};
        uint32_t bv = B, akv = 0;
        if (valid) {
            mine = load_owner<kFilter>(a.P, p);
            bv = static_cast<uint32_t>(a.P.key[p] >> 32);
            akv = a.P.akey[p];
        }
        const uint32_t bmin = __reduce_min_sync(full, bv);
        int queued = 0;
        for (uint32_t i = bmin; i < B; ++i) {
            const uint32_t s = S.start[i], e = S.start[i + 1];
            if (s == e) continue;
            uint32_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;
            if (valid && i >= bv) {
                const uint32_t Wk = kFilter ? window_filter(mine, S, i) : window_fp64(mine, S, i, coshR);
                key_ranges(a.P.akey, s, e, akv, Wk, r0, r1, r2, r3);
                if (i == bv) {  // same band: each pair once, from the smaller position
                    r0 = r0 > p + 1 ? r0 : p + 1;
                    r2 = r2 > p + 1 ? r2 : p + 1;
                }
                if (r1 < r0) r1 = r0;
                if (r3 < r2) r3 = r2;
                cand += (r1 - r0) + (r3 - r2);
                if (r1 - r0 > a.heavy_min) {
                    push_heavy(a, p, r0, r1);
                    r1 = r0;
                }
                if (r3 - r2 > a.heavy_min) {
                    push_heavy(a, p, r2, r3);
                    r3 = r2;
                }
            }
            const int c0 = r1 > r0, c1 = r3 > r2, cnt = c0 + c1;
            int incl = cnt;
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(full, incl, off);
                if (lane >= off) incl += y;
            }
            const int total = __shfl_sync(full, incl, 31);
            if (total == 0) continue;
            if (queued + total > kListCap) {
                flush<kFilter, kCsr>(a, W, queued, mine, coshR, verify, near);
                queued = 0;
            }
            int at = queued + incl - cnt;
            if (c0) {
                W.lo[at] = r0;
                W.hi[at] = r1;
                W.own[at] = lane;
                ++at;
            }
            if (c1) {
                W.lo[at] = r2;
                W.hi[at] = r3;
                W.own[at] = lane;
            }
            queued += total;
            __syncwarp();
        }
        if (queued) flush<kFilter, kCsr>(a, W, queued, mine, coshR, verify, near);
    }
    for (int off = 16; off; off >>= 1) {
        cand += __shfl_down_sync(full, cand, off);
        near += __shfl_down_sync(full, near, off);
    }
    if (lane == 0) {
        if (cand) atomicAdd(reinterpret_cast<unsigned long long *>(&M->candidates), cand);
        if (near) atomicAdd(reinterpret_cast<unsigned long long *>(&M->near_threshold),
                            static_cast<unsigned long long>(near));
    }
}

// Heavy chunks: one warp per chunk of at most kChunk candidates of one owner.
template <bool kFilter, bool kCsr>
__global__ void __launch_bounds__(kThreads) heavy_kernel(QueryArgs a)
{
    __shared__ WarpSmem Wsm[kWarps];
    Meta *M = a.M;
    if (M->error || (M->filter != 0) != kFilter) return;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem &W = Wsm[warp];
    const double coshR = M->coshR;
    const bool verify = M->verify != 0;
    const uint32_t count = M->heavy_n < a.heavy_cap ? M->heavy_n : a.heavy_cap;
    uint32_t near = 0;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&M->heavy_next, 1u);
        item = __shfl_sync(full, item, 0);
        if (item >= count) break;
        const uint4 h = a.heavy[item];
        // every lane holds the owner; the flush broadcasts from lane 0
        const Owner mine = load_owner<kFilter>(a.P, h.x);
        if (lane == 0) {
            W.lo[0] = h.y;
            W.hi[0] = h.z;
            W.own[0] = 0;
        }
        __syncwarp();
        flush<kFilter, kCsr>(a, W, 1, mine, coshR, verify, near);
    }
    for (int off = 16; off; off >>= 1) near += __shfl_down_sync(full, near, off);
    if (lane == 0 && near)
        atomicAdd(reinterpret_cast<unsigned long long *>(&M->near_threshold), static_cast<unsigned long long>(near));
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
    uint32_t near = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; w0 < count; w0 += stride) {
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
            near += fabs(L - coshR) <= 1e-12 * coshR;
        }
        const uint32_t word = __ballot_sync(full, edge);
        if (!word) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long *>(&M->m), __popc(word));
        base = __shfl_sync(full, base, 0);
        if (edge && base + __popc(word) <= a.capacity) write_edge<kCsr>(a, base + __popc(word & lt), idv, idw);
    }
    for (int off = 16; off; off >>= 1) near += __shfl_down_sync(full, near, off);
    if (lane == 0 && near)
        atomicAdd(reinterpret_cast<unsigned long long *>(&M->near_threshold), static_cast<unsigned long long>(near));
    if (blockIdx.x == 0 && threadIdx.x == 0) M->rechecks = count;
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

template <typename K>
int resident_ctas(K kernel)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
    return (per_sm > 0 ? per_sm : 1) * num_sms();
}

template <bool kFilter, bool kCsr>
Status run(const QueryArgs &a, cudaStream_t stream)
{
    Status st;
    const uint64_t nbatch = (a.P.n + 31) / 32;
    const uint64_t need = ceil_div(nbatch ? nbatch : 1, kWarps);
    static int grid_b = 0, grid_h = 0;
    if (!grid_b) grid_b = resident_ctas(batch_kernel<kFilter, kCsr>);
    if (!grid_h) grid_h = resident_ctas(heavy_kernel<kFilter, kCsr>);
    const unsigned gb = static_cast<unsigned>(need < static_cast<uint64_t>(grid_b) ? need : grid_b);
    batch_kernel<kFilter, kCsr><<<gb, kThreads, 0, stream>>>(a);
    RHG_LAUNCH_CHECK();
    heavy_kernel<kFilter, kCsr><<<static_cast<unsigned>(grid_h), kThreads, 0, stream>>>(a);
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
    Status st = csr ? run<true, true>(a, stream) : run<true, false>(a, stream);
    if (st.code) return st;
    return csr ? run<false, true>(a, stream) : run<false, false>(a, stream);
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
