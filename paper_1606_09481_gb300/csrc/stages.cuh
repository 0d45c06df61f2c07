// stages.cuh -- device bodies of the point pipeline's stages that both the
// per-stage kernels and the persistent batch kernel run: the plan (R and band
// boundaries, Sec. III-A/B), sampling (Alg. 1 sampling step, Eq. 1), band
// offsets, the filter values, the stable radix-sort tile pass and the bucket sort
// (Alg. 1, angular sort within each band) with the gather fused in, and the
// per-graph results.  A body that works on one tile, graph or bucket takes its
// index and its shared memory from the caller, so that one CTA can run several
// items one after another.
#pragma once
#include "kernels.h"

namespace rhg {
namespace {
namespace stg {

using dm::add;
using dm::div;
using dm::mul;
using dm::sub;

// Eq. 22 of Krioukov et al. with zeta = 1 (Sec. III-B), in the fixed operation order
// of the deterministic definition:
//   kbar = ((2/pi) xi^2 n) * (e^{-R/2} + e^{-alpha R} ((alpha R / 2) inner - 1)),
//   inner = (pi/4)/alpha^2 - (pi-1)/alpha + (pi-2),  xi = alpha/(alpha - 1/2).
__device__ double kbar(double R, double nd, double alpha)
{
    const double xi = div(alpha, sub(alpha, 0.5));
    const double pre = mul(mul(div(2.0, dm::kPi), mul(xi, xi)), nd);
    const double e1 = dm::exp(-mul(R, 0.5));
    const double e2 = dm::exp(-mul(alpha, R));
    const double ta = mul(mul(dm::kPi, 0.25), div(1.0, mul(alpha, alpha)));
    const double tb = div(sub(dm::kPi, 1.0), alpha);
    const double inner = add(sub(ta, tb), sub(dm::kPi, 2.0));
    const double br = sub(mul(mul(mul(alpha, R), 0.5), inner), 1.0);
    return mul(pre, add(e1, mul(e2, br)));
}

constexpr int kBracket = 256;      // grid points j = 0..255 of the bracket search
constexpr int kPlanThreads = 256;  // the single-graph plan: 8 bisection steps per round
constexpr int kPlanNodes = 256;    // speculative nodes per round, at most (deeper rounds
                                   // are bound by the FP64 pipe's throughput: measured slower)

// Shared state of plan_block.
struct PlanSmem {
    double R_sh, lo_sh, hi_sh, sq;
    int jstar, fail, walk_done;
    double mid[kPlanNodes];      // node t of a round's tree: its midpoint
    uint8_t above[kPlanNodes];   // kbar(its midpoint) > k
    uint8_t valid[kPlanNodes];   // its midpoint lies strictly inside its interval
};

__device__ __forceinline__ bool same(double x, double y)
{
    return __double_as_longlong(x) == __double_as_longlong(y);  // non-negative, finite
}

// R, boundaries and the band constants of one graph, by one CTA.  depth:
// bisection steps taken per round (2^depth - 1 speculative evaluations, at most
// blockDim.x - 1 and kPlanNodes - 1; 8 when one graph wants the lowest latency,
// fewer when many graphs share the FP64 units).  GB300's FP64 pipe takes tens of
// ns per dependent operation, so the work is laid out for short serial chains.
// All threads of the CTA call it (it synchronises the CTA); blockDim.x >= kBracket.
__device__ void plan_block(Meta *M, const PlanArgs &a, int depth, PlanSmem &PS)
{
    int &jstar = PS.jstar;
    double &R_sh = PS.R_sh, &lo_sh = PS.lo_sh, &hi_sh = PS.hi_sh;
    int &fail = PS.fail, &walk_done = PS.walk_done;
    const int t = threadIdx.x;
    const double nd = static_cast<double>(a.n);
    const double alpha = a.alpha, k = a.k;
    if (t == 0) {
        jstar = -1;
        fail = 0;
        R_sh = a.R_override;
    }
    __syncthreads();
    if (!(a.R_override > 0.0)) {
        // bracket: the largest integer grid point j with kbar(j) > k
        if (t < kBracket && kbar(static_cast<double>(t), nd, alpha) > k) atomicMax(&jstar, t);
        __syncthreads();
        if (t == 0) {
            fail = (jstar < 0 || jstar == kBracket - 1) ? 1 : 0;
            walk_done = fail;
            lo_sh = static_cast<double>(jstar);
            hi_sh = static_cast<double>(jstar + 1);
        }
        __syncthreads();
        // binary search: mid = (lo + hi) / 2, kbar(mid) > k ? lo = mid : hi = mid, until
        // lo and hi are adjacent (at most 200 steps); R = hi.  Each round takes
        // `depth` steps at once: thread t (heap order, root 1) replays the path its
        // index spells from (lo, hi), keeps its midpoint and evaluates kbar there;
        // then thread 0 follows the comparisons through the kept midpoints: the
        // same midpoints and decisions as one step at a time.
        const int nodes = 1 << depth;
        int steps = 0;
        for (int round = 0; round < 200; ++round) {
            if (walk_done) break;
            if (t >= 1 && t < nodes) {
                double lo = lo_sh, hi = hi_sh;
                const int level = 31 - __clz(t);
                bool live = true;
                for (int d = level - 1; d >= 0 && live; --d) {
                    const double mid = mul(add(lo, hi), 0.5);
                    if (same(mid, lo) || same(mid, hi)) live = false;
                    else if ((t >> d) & 1) lo = mid;
                    else hi = mid;
                }
                uint8_t b = 0, v = 0;
                if (live) {
                    const double mid = mul(add(lo, hi), 0.5);
                    if (!same(mid, lo) && !same(mid, hi)) {
                        v = 1;
                        PS.mid[t] = mid;
                        b = kbar(mid, nd, alpha) > k ? 1 : 0;
                    }
                }
                PS.above[t] = b;
                PS.valid[t] = v;
            }
            __syncthreads();
            if (t == 0) {
                double lo = lo_sh, hi = hi_sh;
                int node = 1;
                for (int d = 0; d < depth; ++d) {
                    if (!PS.valid[node] || steps == 200) {
                        walk_done = 1;
                        break;
                    }
                    ++steps;
                    if (PS.above[node]) {
                        lo = PS.mid[node];
                        node = 2 * node + 1;
                    } else {
                        hi = PS.mid[node];
                        node = 2 * node;
                    }
                }
                lo_sh = lo;
                hi_sh = hi;
            }
            __syncthreads();
        }
        if (t == 0 && !fail) R_sh = hi_sh;
    }
    __syncthreads();
    const double R = fail ? 1.0 : R_sh;
    const uint32_t B = a.B;
    // e^k table (threads 0..128), cosh R, G, e^-G, the scalars and the boundaries
    // (a short recurrence), each part by its own thread
    if (t <= 2 * kExpTab) M->etab[t] = static_cast<float>(::exp(static_cast<double>(t - kExpTab)));
    if (t == 2 * kExpTab + 1) {
        const double coshR = dm::cosh(R);
        const double G = 0.5 * ::log(2.0 * coshR);
        M->coshR = coshR;
        M->G = G;
        PS.sq = ::exp(-G);
    }
    if (t == 2 * kExpTab + 2) M->cm1 = sub(dm::cosh(mul(alpha, R)), 1.0);
    if (t == 0) {
        M->error = fail ? kErrNoSolution : kErrNone;
        M->R = R;
        M->alpha = alpha;
        M->inv_alpha = div(1.0, alpha);
        const double p = a.p;
        M->B = B;
        M->batch_budget = a.batch_budget;
        M->core_heavy = a.core_heavy;
        M->fringe_limit = a.fringe_limit;
        M->n = a.n;
        M->seed = a.seed;
        M->k = k;
        M->filter = (a.allow_filter && R <= kFilterMaxR && alpha * R <= kFilterMaxAlphaR) ? 1u : 0u;
        M->verify = a.verify;
        // Sec. III-A: c_0 = 0, c_{j+1} - c_j = c_1 p^j, c_1 = (1-p) R / (1 - p^B), c_B = R
        M->c[0] = 0.0;
        if (p == 1.0) {
            for (uint32_t j = 1; j < B; ++j) M->c[j] = div(mul(R, static_cast<double>(j)), static_cast<double>(B));
        } else {
            double pw = 1.0;
            for (uint32_t j = 0; j < B; ++j) pw = mul(pw, p);
            const double c1 = div(mul(sub(1.0, p), R), sub(1.0, pw));
            double step = c1;
            for (uint32_t j = 1; j < B; ++j) {
                const double next = add(M->c[j - 1], step);
                M->c[j] = next < R ? next : R;
                step = mul(step, p);
            }
        }
        M->c[B] = R;
    }
    __syncthreads();
    const double G = M->G, sq = PS.sq, cm1 = M->cm1;
    // per band j: the FP64 cosh / sinh of the boundary and the FP32 window constants
    // (band i is bounded by c_i - kDeltaR (inner) and c_{i+1} + kDeltaR (outer), a
    // slack well above how far a member's FP64 radius can be from its band: 1e-13,
    // band_of_u53; caller points are assigned by their FP64 radius); the variate
    // thresholds band_u (band_of_u53); the exponent tables (filter_values_u53).
    // One value per thread.
    const uint32_t nv = 10 * (B + 1) + 2 * kYTab;
    for (uint32_t v = t; v < nv; v += blockDim.x) {
        if (v < 10 * (B + 1)) {
            const uint32_t j = v / 10, which = v % 10;
            const double cj = M->c[j];
            const double ci = cj - kDeltaR > 0.0 ? cj - kDeltaR : 0.0;
            const double co = (j < B ? M->c[j + 1] : R) + kDeltaR;
            switch (which) {
                case 0: M->cosh_c[j] = ::cosh(cj); break;
                case 1: M->sinh_c[j] = ::sinh(cj); break;
                case 2: M->band_P[j] = static_cast<float>(::exp(ci) * sq); break;
                case 3: M->band_M[j] = static_cast<float>(::exp(-ci) * sq); break;
                case 4: M->band_S[j] = static_cast<float>(::sinh(ci) * sq * 1.4142135623730951); break;
                case 5: M->band_PMn[j] = static_cast<float>(2.0 * ::cosh(co) * sq * (1.0 + 1e-6)); break;
                case 6: M->band_Po[j] = static_cast<float>(::exp(co) * sq); break;
                case 7: M->band_Mo[j] = static_cast<float>(::exp(-co) * sq); break;
                case 8: M->band_So[j] = static_cast<float>(::sinh(co) * sq * 1.4142135623730951); break;
                default: {
                    uint64_t bu = 0;
                    if (j == B) {
                        bu = uint64_t{1} << 53;
                    } else if (j > 0) {
                        const double sh = ::sinh(0.5 * alpha * cj);
                        const double F = 2.0 * sh * sh / cm1;  // (cosh(alpha c_j) - 1) / (cosh(alpha R) - 1)
                        const double T = ceil(F * 9007199254740992.0);
                        bu = T <= 0.0 ? 0 : (T >= 9007199254740992.0 ? uint64_t{1} << 53 : static_cast<uint64_t>(T));
                    }
                    M->band_u[j] = bu;
                }
            }
        } else {
            const uint32_t e = (v - 10 * (B + 1)) >> 1;
            const double ea = static_cast<double>(e) * 0.69314718055994530942 / alpha;  // ln(2^(e/alpha))
            if ((v - 10 * (B + 1)) & 1u) M->tabM[e] = static_cast<float>(::exp(-ea - G));
            else M->tabP[e] = static_cast<float>(fmin(::exp(ea - G), 3.0e38));
        }
    }
    if (t < kMaxBands) M->band_count[t] = 0;
    __syncthreads();  // band_u complete
    // sort buckets: 2^b per band with kBucketTarget <= E / 2^b < 2 kBucketTarget for
    // the band's expected count E = n (F(c_{j+1}) - F(c_j)) (b = 0 below), from
    // integers: E / kBucketTarget = n (band_u[j+1] - band_u[j]) 2^-62, so b is
    // floor(log2) of that product minus 62, clamped to [0, 24]
    if (t < kMaxBands) {
        uint32_t b = 0;
        if (static_cast<uint32_t>(t) < B) {
            const uint64_t du = M->band_u[t + 1] - M->band_u[t];
            const uint64_t lo = a.n * du, hi = __umul64hi(a.n, du);
            const int L = hi ? 127 - __clzll(static_cast<long long>(hi))
                             : (lo ? 63 - __clzll(static_cast<long long>(lo)) : -1);
            b = L > 62 ? (L - 62 > 24 ? 24u : static_cast<uint32_t>(L - 62)) : 0u;
        }
        M->bk_bits[t] = b;
    }
    __syncthreads();
    if (t == 0) {
        uint32_t off = 0;
        for (uint32_t j = 0; j < B; ++j) {
            M->bk_off[j] = off;
            off += 1u << M->bk_bits[j];
        }
        M->bk_off[B] = off;
        M->nbuckets = off;
    }
    __syncthreads();
    if (a.bucket_counts)
        for (uint32_t j = t; j < M->nbuckets; j += blockDim.x) a.bucket_counts[j] = 0;
    if (t != 0) return;
    M->cw = static_cast<float>(cm1 * 0x1.0p-53);
    M->inv_alpha_f = static_cast<float>(1.0 / alpha);
    M->y_one = static_cast<float>(::exp(alpha));
    M->alpha_one = alpha == 1.0 ? 1u : 0u;
    M->m = 0;
    M->candidates = 0;
    M->near_threshold = 0;
    M->rounding_band = 0;
    M->rechecks = 0;
    M->verify_failures = 0;
    M->heavy_n = 0;
    M->heavy_next = 0;
    M->recheck_n = 0;
    M->heavy_lo = 0;
    M->recheck_lo = 0;
    M->work_counter = 0;
    for (uint32_t c = 0; c < kClaimCounters; ++c) M->claim[c * 32] = 0;
}

// Batch, item vb of G + 1 (one CTA each): item g < G plans graph g; item G
// clears the control block's counters.
__device__ void plan_batch_item(Meta *metas, const PlanArgs *args, uint32_t G, uint32_t vb, PlanSmem &PS)
{
    if (vb < G) {
        const PlanArgs a = args[vb];
        plan_block(metas + vb, a, 5, PS);
        return;
    }
    if (threadIdx.x != 0) return;
    Meta *C = metas + G;
    C->error = kErrNone;
    C->filter = 0;
    C->verify = 0;
    C->m = 0;
    C->candidates = 0;
    C->near_threshold = 0;
    C->rounding_band = 0;
    C->rechecks = 0;
    C->verify_failures = 0;
    C->heavy_n = 0;
    C->heavy_next = 0;
    C->recheck_n = 0;
    C->heavy_lo = 0;
    C->recheck_lo = 0;
    C->work_counter = 0;
    for (uint32_t c = 0; c < kClaimCounters; ++c) C->claim[c * 32] = 0;
}


constexpr int kSampleThreads = 256;

struct SampleSmem {
    double c[kMaxBands + 1];
    uint64_t bu[kMaxBands + 1];
    uint32_t bk_off[kMaxBands + 1], bk_bits[kMaxBands];
    unsigned int hist[kMaxBands];
};

// Adds the warp's points to the band histogram: one shared atomic per distinct
// band among the lanes (b = kMaxBands for a lane without a point).  All lanes call it.
__device__ __forceinline__ void hist_add_warp(unsigned int *hist, uint32_t b)
{
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const unsigned lane = threadIdx.x & 31u;
    if (b < static_cast<uint32_t>(kMaxBands) && (peers & ((1u << lane) - 1u)) == 0)
        atomicAdd(&hist[b], static_cast<unsigned int>(__popc(peers)));
}

// Batch, tile t (one CTA): position p of graph g holds vertex p - pt_off[g]; the
// FP64 radius (FP64 mode) is stored by position.
__device__ void sample_tile(Meta *metas, const BatchTables &bt, uint64_t *keys, double *r_by_pos, uint32_t *bk_counts,
                            uint32_t t, SampleSmem &SS)
{
    double *c = SS.c;
    uint64_t *bu = SS.bu;
    unsigned int *hist = SS.hist;
    __syncthreads();  // the CTA's previous item is done with the shared arrays
    const uint4 T = bt.tiles[t];
    Meta *M = metas + T.x;
    const uint32_t B = M->B;
    const bool filter = M->filter != 0;
    const double R = M->R, cm1 = M->cm1, inv_alpha = M->inv_alpha;
    const uint64_t seed = M->seed;
    if (threadIdx.x <= B) {
        c[threadIdx.x] = M->c[threadIdx.x];
        bu[threadIdx.x] = M->band_u[threadIdx.x];
        SS.bk_off[threadIdx.x] = M->bk_off[threadIdx.x];
        if (threadIdx.x < B) SS.bk_bits[threadIdx.x] = M->bk_bits[threadIdx.x];
    }
    if (threadIdx.x < kMaxBands) hist[threadIdx.x] = 0;
    __syncthreads();
    if (M->error) return;
    const uint32_t first_id = T.y - bt.pt_off[T.x];
    uint32_t *counts = bk_counts + bt.bk_base[T.x];
    // warp-uniform trip count (the histograms are counted per warp)
    for (uint32_t j0 = threadIdx.x & ~31u; j0 < T.z; j0 += blockDim.x) {
        const uint32_t j = j0 + (threadIdx.x & 31u);
        uint32_t b = kMaxBands, akey = 0;
        if (j < T.z) {
            const uint32_t id = first_id + j, pos = T.y + j;
            const U64x4 x = draw(id, seed);
            akey = static_cast<uint32_t>(x.x0 >> 32);
            if (filter) {
                b = band_of_u53(x.x1 >> 11, bu, B);
            } else {
                const double r = radius_from_u53(x.x1 >> 11, R, cm1, inv_alpha);
                r_by_pos[pos] = r;
                b = band_of(r, c, B);
            }
            keys[pos] = (static_cast<uint64_t>(b) << 32) | akey;
        }
        hist_add_warp(hist, b);
        const uint32_t bk = b < B ? bucket_of((static_cast<uint64_t>(b) << 32) | akey, SS.bk_off, SS.bk_bits)
                                  : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, bk);
        if (bk != 0xffffffffu && (peers & ((1u << (threadIdx.x & 31u)) - 1u)) == 0)
            atomicAdd(&counts[bk], static_cast<uint32_t>(__popc(peers)));
    }
    __syncthreads();
    if (threadIdx.x < B && hist[threadIdx.x]) atomicAdd(&M->band_count[threadIdx.x], hist[threadIdx.x]);
}

// Band starts (sorted positions) and bucket-index offsets of one graph whose
// positions start at pos0 and whose index entries start at idx0.
__device__ void band_offsets_one(Meta *M, uint64_t pos0, uint32_t idx0)
{
    uint64_t s = pos0;
    uint32_t off = idx0;
    for (uint32_t j = 0; j < M->B; ++j) {
        M->band_start[j] = s;
        s += M->band_count[j];
        // 2^b buckets, the largest power of two <= count / kBucketPoints, b >= 1
        uint32_t b = 1;
        while (b < 31 && (uint64_t{2} << b) * kBucketPoints <= M->band_count[j]) ++b;
        M->idx_off[j] = off;
        M->idx_shift[j] = 32 - b;
        off += (1u << b) + 1;
    }
    M->band_start[M->B] = s;
    M->idx_off[M->B] = off;
}

// e^x in FP32 with relative error <= 4 * 2^-24 for |x| <= kExpTab + 1/2:
// x = k + f with integer k, |f| <= 1/2 exact in FP64, e^k from the table.
__device__ __forceinline__ float exp_split(double x, const float *etab)
{
    const double kd = rint(x);
    const int k = static_cast<int>(kd);
    const float f = static_cast<float>(x - kd);
    return etab[k + kExpTab] * expf(f);
}

// Filter-mode values of a point from its FP64 angle and (approximate) radius.
__device__ __forceinline__ void filter_values(double ph, double r, double G, const float *etab, float2 *ang,
                                              float4 *pms)
{
    const float hi = static_cast<float>(ph);
    const float lo = static_cast<float>(ph - static_cast<double>(hi));
    *ang = make_float2(hi, lo);
    const float P = exp_split(r - G, etab);
    const float Mv = exp_split(-r - G, etab);
    float S, gam;
    if (r >= 1.0) {
        S = (P - Mv) * 0.70710678118654752f;
        gam = kEpsPM * ((P + Mv) / (P - Mv)) + 2.0f * kEps32;
    } else if (r > 0.0) {
        S = static_cast<float>(::sinh(r) * ::exp(-G) * 1.4142135623730951);
        gam = kEpsPM * static_cast<float>(::cosh(r) / ::sinh(r)) + 2.0f * kEps32;
    } else {
        S = 0.0f;
        gam = 0.0f;
    }
    *pms = make_float4(P, Mv, S, gam);
}

// Per-graph constants of filter_values_u53, staged in shared memory.
struct YTab {
    float P[kYTab], M[kYTab];
    float cw, ia, y_one;
    uint32_t alpha_one;
    double G, inv_alpha;
};

// All threads call it; the caller synchronises before the first use.
__device__ __forceinline__ void load_ytab(YTab &Y, const Meta *M)
{
    for (int j = threadIdx.x; j < kYTab; j += blockDim.x) {
        Y.P[j] = M->tabP[j];
        Y.M[j] = M->tabM[j];
    }
    if (threadIdx.x == 0) {
        Y.cw = M->cw;
        Y.ia = M->inv_alpha_f;
        Y.y_one = M->y_one;
        Y.alpha_one = M->alpha_one;
        Y.G = M->G;
        Y.inv_alpha = M->inv_alpha;
    }
}

// The same constants where filter_values_u53 reads them: shared memory (YTab) or
// a graph's Meta in global memory.
struct YRef {
    const float *P, *M;
    float cw, ia, y_one;
    uint32_t alpha_one;
    double G, inv_alpha;
};
__device__ __forceinline__ YRef yref(const YTab &Y)
{
    return YRef{Y.P, Y.M, Y.cw, Y.ia, Y.y_one, Y.alpha_one, Y.G, Y.inv_alpha};
}
__device__ __forceinline__ YRef yref(const Meta *M)
{
    return YRef{M->tabP, M->tabM, M->cw, M->inv_alpha_f, M->y_one, M->alpha_one, M->G, M->inv_alpha};
}

// Filter-mode values of a generated point from its variates (ua: angle, ur:
// radius), in FP32 and integer arithmetic (the rare points with r < 1 aside):
//   angle  angle_hilo_u53: the pair filter_values forms from the FP64 angle;
//   y      w = U (cosh(alpha R) - 1) as fl(fl(U) cw) (relative error <= 3 u,
//          u = 2^-24), y = (1 + w) + sqrt(w (w + 2)) in FP32: within 6 u of the
//          exact y = e^{alpha r} (dy/y = dw / sqrt(w^2 + 2 w) <= dw/w, and three
//          roundings of positive terms);
//   P, M   y = 2^e m with m in [sqrt(1/2), sqrt(2)): e^{r - G} = y^{1/alpha} e^{-G}
//          = tabP[e] m^{1/alpha}, e^{-r-G} = tabM[e] m^{-1/alpha}; m^{+-1/alpha} is
//          m and 1/m for alpha = 1, else exp2f(+-log2f(m) / alpha) (log2f within
//          1 ulp, exp2f within 2 ulp: <= 3.7e-7 relative); with the rounding of the
//          table entry and of the product the relative error is <= 6 u / alpha +
//          3.7e-7 + 2 u <= 1.2e-6 < kEpsPM for alpha > 1/2;
//   S      (P - M) / sqrt 2 for r >= 1 (y >= e^alpha), as filter_values; below,
//          from the radius ln(y) / alpha in FP64 (absolute error <= 6 u / alpha).
__device__ __forceinline__ void filter_values_u53(uint64_t ua, uint64_t ur, const YRef &Y, float2 *ang,
                                                  float4 *pms)
{
    *ang = angle_hilo_u53(ua);
    const float wf = u53_to_float(ur) * Y.cw;
    const float y = (1.0f + wf) + sqrtf(wf * (wf + 2.0f));
    const int bits = __float_as_int(y);  // y >= 1: normal
    int e = (bits >> 23) - 126;
    float m = __int_as_float((bits & 0x007fffff) | 0x3f000000);  // y = 2^e m, m in [1/2, 1)
    if (m < 0.70710678f) {
        m *= 2.0f;
        e -= 1;
    }
    e = e < 0 ? 0 : (e >= kYTab ? kYTab - 1 : e);
    float mp, mm;
    if (Y.alpha_one) {
        mp = m;
        mm = 1.0f / m;
    } else {
        const float t = log2f(m) * Y.ia;
        mp = exp2f(t);
        mm = exp2f(-t);
    }
    const float P = Y.P[e] * mp;
    const float Mv = Y.M[e] * mm;
    float S, gam;
    if (y >= Y.y_one) {
        S = (P - Mv) * 0.70710678118654752f;
        gam = kEpsPM * ((P + Mv) / (P - Mv)) + 2.0f * kEps32;
    } else if (y > 1.0f) {
        const double r = ::log(static_cast<double>(y)) * Y.inv_alpha;
        S = static_cast<float>(::sinh(r) * ::exp(-Y.G) * 1.4142135623730951);
        gam = kEpsPM * static_cast<float>(::cosh(r) / ::sinh(r)) + 2.0f * kEps32;
    } else {
        S = 0.0f;
        gam = 0.0f;
    }
    *pms = make_float4(P, Mv, S, gam);
}

// Per-graph results of a batch: {m low, m high, R low, R high} and {B, error}.
__device__ void batch_result_one(const Meta *metas, uint32_t g, uint4 *out)
{
    const Meta *M = metas + g;
    const uint64_t m = M->m;
    const uint64_t Rb = static_cast<uint64_t>(__double_as_longlong(M->R));
    out[2 * g] = make_uint4(static_cast<uint32_t>(m), static_cast<uint32_t>(m >> 32), static_cast<uint32_t>(Rb),
                            static_cast<uint32_t>(Rb >> 32));
    out[2 * g + 1] = make_uint4(M->B, M->error, M->filter, 0u);
}


// ---- radix sort (stable LSD, 8-bit digits)
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // keys per tile
constexpr int kRadix = 256;

struct TileSmem {
    uint32_t digit_base[kRadix];  // output position of the next key of each digit
    uint32_t warp_count[kWarps][kRadix];
    uint32_t tile_start[kRadix];
    uint32_t warp_sum[kWarps];
    uint64_t skey[kTile];
};

// Exclusive scan of one value per thread over the CTA (kThreads = 8 warps);
// warp_sum is scratch.  Ends with a barrier.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t *warp_sum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += warp_sum[w];
    __syncthreads();
    return before + incl - v;
}

// One tile [tile, tile + cnt) of a pass: every warp ranks its 32 x kItems keys
// with __match_any_sync, warps are combined by a per-digit prefix over warps, so
// the order of equal digits is the input order (stable); the tile is staged in
// shared memory in digit order and written out from there, one contiguous run
// per digit, at sm.digit_base (which then advances by the tile's counts).
template <bool kValues>
__device__ __forceinline__ void tile_pass(const uint64_t *keys_in, uint64_t *keys_out, const uint32_t *vals_in,
                                          uint32_t *vals_out, uint64_t tile, uint32_t cnt, int shift, TileSmem &sm,
                                          uint32_t *sval)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    for (int w = 0; w < kWarps; ++w) sm.warp_count[w][threadIdx.x] = 0;
    __syncthreads();
    // rank within the warp's sub-tile: element (i, lane) = i*32 + lane of the sub-tile
    const uint32_t sub = static_cast<uint32_t>(warp) * 32 * kItems;
    uint64_t key[kItems];
    uint32_t val[kItems];
    uint32_t rank[kItems];
    int digit[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t local = sub + static_cast<uint32_t>(i) * 32 + lane;
        const bool valid = local < cnt;
        key[i] = valid ? keys_in[tile + local] : 0;
        if (kValues) val[i] = valid ? vals_in[tile + local] : 0;
        digit[i] = static_cast<int>((key[i] >> shift) & (kRadix - 1));
        const uint32_t active = __ballot_sync(0xffffffffu, valid);
        rank[i] = 0xffffffffu;
        if (valid) {
            const uint32_t peers = __match_any_sync(active, digit[i]);
            const uint32_t base = sm.warp_count[warp][digit[i]];
            rank[i] = base + __popc(peers & lanemask_lt);
            __syncwarp(active);
            if ((peers & lanemask_lt) == 0) sm.warp_count[warp][digit[i]] = base + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps and the tile total; the digits'
    // starts in the tile are the exclusive scan of the totals
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = sm.warp_count[w][d];
        sm.warp_count[w][d] = run;
        run += c;
    }
    sm.tile_start[d] = block_exclusive(run, sm.warp_sum);
    __syncthreads();
    // the tile in digit order (stable) in shared memory ...
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (rank[i] != 0xffffffffu) {
            const uint32_t local = sm.tile_start[digit[i]] + sm.warp_count[warp][digit[i]] + rank[i];
            sm.skey[local] = key[i];
            if (kValues) sval[local] = val[i];
        }
    }
    __syncthreads();
    // ... then written out in that order: each digit's keys land on consecutive
    // positions, so neighbouring threads write neighbouring addresses
    for (uint32_t j = threadIdx.x; j < cnt; j += kThreads) {
        const uint64_t k = sm.skey[j];
        const int dg = static_cast<int>((k >> shift) & (kRadix - 1));
        const uint32_t pos = sm.digit_base[dg] + (j - sm.tile_start[dg]);
        keys_out[pos] = k;
        if (kValues) vals_out[pos] = sval[j];
    }
    __syncthreads();
    sm.digit_base[d] += run;
    __syncthreads();
}

// ---- bucket sort of generated points (one bucket per call; see bucket.cu)
constexpr uint32_t kSubMax = 32;  // largest sub-bucket sorted by one thread

// LSD radix sort of comp[s, s + cnt) by one CTA (8 passes of 8 bits through
// scratch, tiles in order, so stable), for buckets the shared-memory path cannot
// take.  The result is back in comp.
__device__ void cta_sort_range(uint64_t *comp, uint64_t *scratch, uint32_t s, uint32_t cnt, TileSmem &ts,
                               uint32_t *hist)
{
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        const uint64_t *src = (pass & 1) ? scratch : comp;
        uint64_t *dst = (pass & 1) ? comp : scratch;
        __syncthreads();
        hist[threadIdx.x] = 0;
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < cnt; k += kThreads) atomicAdd(&hist[(src[s + k] >> shift) & 255u], 1u);
        __syncthreads();
        ts.digit_base[threadIdx.x] = s + block_exclusive(hist[threadIdx.x], ts.warp_sum);
        __syncthreads();
        for (uint32_t t = 0; t < cnt; t += kTile) {
            const uint32_t c = cnt - t < static_cast<uint32_t>(kTile) ? cnt - t : kTile;
            tile_pass<false>(src, dst, nullptr, nullptr, s + t, c, shift, ts, nullptr);
        }
    }
    __syncthreads();
}

struct BucketSmem {
    union {
        uint64_t buf[2][kBucketCap];
        TileSmem ts;
    } u;
    uint32_t hist[256], cur[256], wsum[kWarps];
    int big;
};

// Sorts the bucket comp[s, s + cnt), composites (angle key << 32 | id), by
// (angle key, id): in shared memory a counting pass on the 8 angle-key bits at
// composite shift dsh (the ones below the bucket's own), then every sub-bucket by
// one thread (insertion sort); a bucket above kBucketCap, or with a sub-bucket
// above kSubMax, by cta_sort_range in global memory.  Returns where element k of
// the sorted bucket is (shared memory, or comp + s).  All threads of the CTA
// (kThreads) call it; it begins and ends with a barrier.
__device__ const uint64_t *sort_bucket(uint64_t *comp, uint64_t *scratch, uint32_t s, uint32_t cnt, int dsh,
                                       BucketSmem &B)
{
    const uint32_t t = threadIdx.x;
    __syncthreads();  // the CTA's previous bucket is done with B
    if (cnt <= kBucketCap) {
        B.hist[t] = 0;
        if (t == 0) B.big = 0;
        __syncthreads();
        for (uint32_t k = t; k < cnt; k += kThreads) {
            const uint64_t v = comp[s + k];
            B.u.buf[0][k] = v;
            atomicAdd(&B.hist[static_cast<uint32_t>(v >> dsh) & 255u], 1u);
        }
        __syncthreads();
        const uint32_t h = B.hist[t];
        B.cur[t] = block_exclusive(h, B.wsum);
        if (h > kSubMax) B.big = 1;
        __syncthreads();
        for (uint32_t k = t; k < cnt; k += kThreads) {
            const uint64_t v = B.u.buf[0][k];
            B.u.buf[1][atomicAdd(&B.cur[static_cast<uint32_t>(v >> dsh) & 255u], 1u)] = v;
        }
        __syncthreads();
        const bool big = B.big != 0;
        if (!big) {  // sub-bucket t is [cur[t] - h, cur[t])
            uint64_t *x = B.u.buf[1];
            const uint32_t e1 = B.cur[t], s1 = e1 - h;
            for (uint32_t i = s1 + 1; i < e1; ++i) {
                const uint64_t v = x[i];
                uint32_t j = i;
                while (j > s1 && x[j - 1] > v) {
                    x[j] = x[j - 1];
                    --j;
                }
                x[j] = v;
            }
        }
        __syncthreads();
        if (!big) return B.u.buf[1];
    }
    cta_sort_range(comp, scratch, s, cnt, B.u.ts, B.hist);
    return comp + s;
}

// Batch, graph g (one CTA): band offsets (band_offsets_one), then the exclusive
// scan of the graph's bucket counts into bucket starts (global positions) and
// scatter cursors; start[nb] = the graph's end.
__device__ void bucket_scan_graph(Meta *metas, const BatchTables &bt, uint32_t *bk_counts, uint32_t *bk_start,
                                  uint32_t *bk_info, uint32_t g, uint32_t *warp_sum)
{
    __syncthreads();  // the CTA's previous item is done with warp_sum
    Meta *M = metas + g;
    if (threadIdx.x == 0) band_offsets_one(M, bt.pt_off[g], bt.idx_base[g]);
    const uint32_t nb = M->nbuckets, base = bt.bk_base[g], B = M->B;
    const bool bad = M->error != 0;
    uint32_t carry = bt.pt_off[g];
    for (uint32_t j0 = 0; j0 < nb; j0 += kThreads) {
        const uint32_t j = j0 + threadIdx.x;
        const uint32_t v = j < nb && !bad ? bk_counts[base + j] : 0u;
        const uint32_t excl = block_exclusive(v, warp_sum);  // ends with a barrier
        uint32_t chunk = 0;
        for (int w = 0; w < kWarps; ++w) chunk += warp_sum[w];
        if (j < nb) {
            bk_start[base + j] = carry + excl;
            bk_counts[base + j] = carry + excl;
            uint32_t band = 0;  // the largest band whose first bucket is <= j
            for (uint32_t step = 32; step; step >>= 1)
                if (band + step < B && M->bk_off[band + step] <= j) band += step;
            bk_info[base + j] = (g << 6) | band;  // a graph in error has only empty buckets
        }
        carry += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) bk_start[base + nb] = carry;
    // the graph's unused bucket slots
    for (uint32_t j = nb + threadIdx.x; j < bt.bk_base[g + 1] - base; j += kThreads) bk_info[base + j] = 0xffffffffu;
}

// Batch, tile t (one CTA): each point's composite (angle key << 32 | id) to its
// bucket, at a cursor taken with an atomic add.
__device__ void bucket_scatter_tile(const Meta *metas, const BatchTables &bt, const uint64_t *keys, uint32_t *cursor,
                                    uint64_t *comp, uint32_t t, uint32_t *off, uint32_t *bits)
{
    __syncthreads();  // the CTA's previous item is done with the tables
    const uint4 T = bt.tiles[t];
    const Meta *M = metas + T.x;
    const uint32_t B = M->B;
    if (threadIdx.x <= B) {
        off[threadIdx.x] = M->bk_off[threadIdx.x];
        if (threadIdx.x < B) bits[threadIdx.x] = M->bk_bits[threadIdx.x];
    }
    __syncthreads();
    if (M->error) return;
    uint32_t *cur = cursor + bt.bk_base[T.x];
    const uint32_t first_id = T.y - bt.pt_off[T.x];
    for (uint32_t j = threadIdx.x; j < T.z; j += blockDim.x) {
        const uint64_t k = keys[T.y + j];
        comp[atomicAdd(&cur[bucket_of(k, off, bits)], 1u)] = (k << 32) | (first_id + j);
    }
}

// Batch, one bucket (one CTA): info = graph << 6 | band, the bucket's points
// [s, s + cnt); the bucket sorted (sort_bucket), then the sorted key back into
// comp (P.key) and each point's arrays, as the single-graph bucket sort writes
// them (ids are the graph's own, the FP64 radius by position).
__device__ void bucket_gather_item(Meta *metas, const BatchTables &bt, uint32_t info, uint32_t s, uint32_t cnt,
                                   uint64_t *comp, uint64_t *scratch, const double *r_by_pos, const SortedPoints &P,
                                   BucketSmem &SB)
{
    const uint32_t g = info >> 6, band = info & 63u;
    const Meta *M = metas + g;
    const int rest = 32 - static_cast<int>(M->bk_bits[band]);
    const int dsh = 32 + (rest > 8 ? rest - 8 : 0);
    const uint64_t *sorted = sort_bucket(comp, scratch, s, cnt, dsh, SB);
    const bool filter = M->filter != 0;
    const uint64_t seed = M->seed;
    const YRef Y = yref(M);
    const uint32_t pos0 = bt.pt_off[g];
    for (uint32_t k = threadIdx.x; k < cnt; k += kThreads) {
        const uint64_t c = sorted[k];
        const uint32_t p = s + k, id = static_cast<uint32_t>(c), akey = static_cast<uint32_t>(c >> 32);
        comp[p] = (static_cast<uint64_t>(band) << 32) | akey;
        P.akey[p] = akey;
        P.id[p] = id;
        const U64x4 x = draw(id, seed);
        if (filter) {
            float2 ang;
            float4 pms;
            filter_values_u53(x.x0 >> 11, x.x1 >> 11, Y, &ang, &pms);
            P.ang[p] = ang;
            P.pms[p] = pms;
        } else {
            const double r = r_by_pos[pos0 + id];
            P.phi[p] = phi_from_u53(x.x0 >> 11);
            P.r[p] = r;
            P.ch[p] = dm::cosh(r);
            P.sh[p] = dm::sinh(r);
        }
    }
}

}  // namespace stg
}  // namespace
}  // namespace rhg
