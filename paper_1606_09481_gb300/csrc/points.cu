// points.cu -- the point pipeline: disk radius R (Sec. III-B getTargetRadius),
// band boundaries (Sec. III-A), Philox sampling of (phi, r) by inverse CDF
// (Alg. 1 sampling step, Eq. 1), band assignment (Alg. 1 band insertion)
// and the gather of the (band, angle)-sorted structure-of-arrays.
#include "kernels.h"

namespace rhg {
namespace {

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

constexpr int kPlanThreads = 256;  // grid points j = 0..255 of the bracket search

// R, boundaries and the band constants of one graph, by one CTA of kPlanThreads.
// depth: bisection steps taken per round (2^depth - 1 speculative evaluations;
// 8 when one graph wants the lowest latency, fewer when many graphs share the
// FP64 units).
__device__ void plan_block(Meta *M, const PlanArgs &a, int depth)
{
    __shared__ int jstar;
    __shared__ double R_sh, lo_sh, hi_sh;
    __shared__ int fail, walk_done;
    __shared__ uint8_t above[kPlanThreads];  // node t of a round's tree: kbar(its midpoint) > k
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
        if (kbar(static_cast<double>(t), nd, alpha) > k) atomicMax(&jstar, t);
        __syncthreads();
        if (t == 0) {
            fail = (jstar < 0 || jstar == kPlanThreads - 1) ? 1 : 0;
            walk_done = fail;
            lo_sh = static_cast<double>(jstar);
            hi_sh = static_cast<double>(jstar + 1);
        }
        __syncthreads();
        // binary search: mid = (lo + hi) / 2, kbar(mid) > k ? lo = mid : hi = mid, until
        // lo and hi are adjacent (at most 200 steps); R = hi.  Each round takes
        // `depth` steps at once: thread t (heap order, root 1) replays the path its
        // index spells from (lo, hi) and evaluates kbar at its midpoint, then thread
        // 0 follows the comparisons: the same midpoints and decisions as one step
        // at a time.
        const int nodes = 1 << depth;
        int steps = 0;
        for (int round = 0; round < 200; ++round) {
            if (walk_done) break;
            if (t >= 1 && t < nodes) {
                double lo = lo_sh, hi = hi_sh;
                const int depth = 31 - __clz(t);
                bool live = true;
                for (int d = depth - 1; d >= 0 && live; --d) {
                    const double mid = mul(add(lo, hi), 0.5);
                    if (mid == lo || mid == hi) live = false;
                    else if ((t >> d) & 1) lo = mid;
                    else hi = mid;
                }
                uint8_t b = 0;
                if (live) {
                    const double mid = mul(add(lo, hi), 0.5);
                    if (mid != lo && mid != hi) b = kbar(mid, nd, alpha) > k ? 1 : 0;
                }
                above[t] = b;
            }
            __syncthreads();
            if (t == 0) {
                double lo = lo_sh, hi = hi_sh;
                int node = 1;
                for (int d = 0; d < depth; ++d) {
                    const double mid = mul(add(lo, hi), 0.5);
                    if (mid == lo || mid == hi || steps == 200) {
                        walk_done = 1;
                        break;
                    }
                    ++steps;
                    if (above[node]) {
                        lo = mid;
                        node = 2 * node + 1;
                    } else {
                        hi = mid;
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
    const double coshR = dm::cosh(R);
    const double G = 0.5 * ::log(2.0 * coshR);
    // e^k table (threads 0..128)
    if (t <= 2 * kExpTab) M->etab[t] = static_cast<float>(::exp(static_cast<double>(t - kExpTab)));
    const uint32_t B = a.B;
    if (t == 0) {  // scalars and the boundaries (a short recurrence)
        M->error = fail ? kErrNoSolution : kErrNone;
        M->R = R;
        M->coshR = coshR;
        M->G = G;
        M->alpha = alpha;
        M->inv_alpha = div(1.0, alpha);
        M->cm1 = sub(dm::cosh(mul(alpha, R)), 1.0);
        const double p = a.p;
        M->B = B;
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
    // FP32 window constants, one band per thread: the filter's radii carry an error
    // up to kDeltaR, so band i is bounded by c_i - kDeltaR (inner) and c_{i+1} +
    // kDeltaR (outer)
    const double sq = ::exp(-G);
    for (uint32_t j = t; j <= B; j += blockDim.x) {
        M->cosh_c[j] = ::cosh(M->c[j]);
        M->sinh_c[j] = ::sinh(M->c[j]);
        const double ci = M->c[j] - kDeltaR > 0.0 ? M->c[j] - kDeltaR : 0.0;
        M->band_P[j] = static_cast<float>(::exp(ci) * sq);
        M->band_M[j] = static_cast<float>(::exp(-ci) * sq);
        M->band_S[j] = static_cast<float>(::sinh(ci) * sq * 1.4142135623730951);
        const double co = (j < B ? M->c[j + 1] : R) + kDeltaR;
        M->band_PMn[j] = static_cast<float>(2.0 * ::cosh(co) * sq * (1.0 + 1e-6));
        M->band_Po[j] = static_cast<float>(::exp(co) * sq);
        M->band_Mo[j] = static_cast<float>(::exp(-co) * sq);
        M->band_So[j] = static_cast<float>(::sinh(co) * sq * 1.4142135623730951);
    }
    if (t < kMaxBands) M->band_count[t] = 0;
    if (t != 0) return;
    M->m = 0;
    M->candidates = 0;
    M->near_threshold = 0;
    M->rounding_band = 0;
    M->rechecks = 0;
    M->verify_failures = 0;
    M->heavy_n = 0;
    M->heavy_next = 0;
    M->recheck_n = 0;
    M->work_counter = 0;
    for (uint32_t c = 0; c < kClaimCounters; ++c) M->claim[c * 32] = 0;
}

__global__ void __launch_bounds__(kPlanThreads) plan_kernel(Meta *M, PlanArgs a) { plan_block(M, a, 8); }

// Batch: CTA g < G plans graph g; CTA G clears the control block's counters.
__global__ void __launch_bounds__(kPlanThreads) plan_batch_kernel(Meta *metas, const PlanArgs *args, uint32_t G)
{
    if (blockIdx.x < G) {
        const PlanArgs a = args[blockIdx.x];
        plan_block(metas + blockIdx.x, a, 3);
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
    C->work_counter = 0;
    for (uint32_t c = 0; c < kClaimCounters; ++c) C->claim[c * 32] = 0;
}

constexpr int kSampleThreads = 256;

// Points by id: sort key (band << 32 | angle key) and id.  In filter mode the band
// comes from the approximate radius (bands are then bounded by c_i -+ kDeltaR);
// otherwise from the FP64 radius, which is also stored by id for the gather.
__global__ void __launch_bounds__(kSampleThreads) sample_kernel(Meta *M, uint64_t n, uint64_t seed,
                                                                uint64_t *keys, uint32_t *ids,
                                                                double *r_by_id)
{
    __shared__ double c[kMaxBands + 1];
    __shared__ unsigned int hist[kMaxBands];
    const uint32_t B = M->B;
    const bool filter = M->filter != 0;
    const double R = M->R, cm1 = M->cm1, inv_alpha = M->inv_alpha;
    if (threadIdx.x <= B) c[threadIdx.x] = M->c[threadIdx.x];
    if (threadIdx.x < kMaxBands) hist[threadIdx.x] = 0;
    __syncthreads();
    if (M->error) return;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const U64x4 x = draw(i, seed);
        double r;
        if (filter) {
            r = radius_approx(x.x1 >> 11, R, cm1, inv_alpha);
        } else {
            r = radius_from_u53(x.x1 >> 11, R, cm1, inv_alpha);
            r_by_id[i] = r;
        }
        const uint32_t b = band_of(r, c, B);
        keys[i] = (static_cast<uint64_t>(b) << 32) | static_cast<uint32_t>(x.x0 >> 32);
        ids[i] = static_cast<uint32_t>(i);
        atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < B && hist[threadIdx.x]) atomicAdd(&M->band_count[threadIdx.x], hist[threadIdx.x]);
}

__global__ void __launch_bounds__(kSampleThreads) load_points_kernel(Meta *M, uint64_t n,
                                                                     const double *phi,
                                                                     const double *rr,
                                                                     uint64_t *keys, uint32_t *ids)
{
    __shared__ double c[kMaxBands + 1];
    __shared__ unsigned int hist[kMaxBands];
    const uint32_t B = M->B;
    const double R = M->R;
    if (threadIdx.x <= B) c[threadIdx.x] = M->c[threadIdx.x];
    if (threadIdx.x < kMaxBands) hist[threadIdx.x] = 0;
    __syncthreads();
    bool bad = false;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const double ph = phi[i], r = rr[i];
        if (!(ph >= 0.0 && ph < dm::kTwoPi && r >= 0.0 && r <= R)) bad = true;
        const uint32_t b = band_of(r >= 0.0 ? r : 0.0, c, B);
        keys[i] = (static_cast<uint64_t>(b) << 32) | angle_key(ph >= 0.0 ? ph : 0.0);
        ids[i] = static_cast<uint32_t>(i);
        atomicAdd(&hist[b], 1u);
    }
    if (bad) atomicMax(&M->error, kErrBadPoint);
    __syncthreads();
    if (threadIdx.x < B && hist[threadIdx.x]) atomicAdd(&M->band_count[threadIdx.x], hist[threadIdx.x]);
}

// Batch: CTA per tile.  Position p of graph g holds vertex p - pt_off[g]; the
// FP64 radius (FP64 mode) is stored by position.
__global__ void __launch_bounds__(kSampleThreads) sample_batch_kernel(Meta *metas, BatchTables bt, uint64_t *keys,
                                                                      uint32_t *ids, double *r_by_pos)
{
    __shared__ double c[kMaxBands + 1];
    __shared__ unsigned int hist[kMaxBands];
    const uint4 T = bt.tiles[blockIdx.x];
    Meta *M = metas + T.x;
    const uint32_t B = M->B;
    const bool filter = M->filter != 0;
    const double R = M->R, cm1 = M->cm1, inv_alpha = M->inv_alpha;
    const uint64_t seed = M->seed;
    if (threadIdx.x <= B) c[threadIdx.x] = M->c[threadIdx.x];
    if (threadIdx.x < kMaxBands) hist[threadIdx.x] = 0;
    __syncthreads();
    if (M->error) return;
    const uint32_t first_id = T.y - bt.pt_off[T.x];
    for (uint32_t j = threadIdx.x; j < T.z; j += blockDim.x) {
        const uint32_t id = first_id + j, pos = T.y + j;
        const U64x4 x = draw(id, seed);
        double r;
        if (filter) {
            r = radius_approx(x.x1 >> 11, R, cm1, inv_alpha);
        } else {
            r = radius_from_u53(x.x1 >> 11, R, cm1, inv_alpha);
            r_by_pos[pos] = r;
        }
        const uint32_t b = band_of(r, c, B);
        keys[pos] = (static_cast<uint64_t>(b) << 32) | static_cast<uint32_t>(x.x0 >> 32);
        ids[pos] = id;
        atomicAdd(&hist[b], 1u);
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

__global__ void band_offsets_kernel(Meta *M)
{
    if (threadIdx.x == 0) band_offsets_one(M, 0, 0);
}

__global__ void band_offsets_batch_kernel(Meta *metas, BatchTables bt)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < bt.G) band_offsets_one(metas + g, bt.pt_off[g], bt.idx_base[g]);
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

__global__ void __launch_bounds__(256) gather_filter_kernel(const Meta *M, uint64_t n, uint64_t seed,
                                                            const uint64_t *keys, const uint32_t *sids,
                                                            const double *phi_src, const double *r_src,
                                                            SortedPoints P)
{
    __shared__ float etab[2 * kExpTab + 1];
    for (int j = threadIdx.x; j <= 2 * kExpTab; j += blockDim.x) etab[j] = M->etab[j];
    __syncthreads();
    if (M->error || !M->filter) return;
    const double G = M->G, R = M->R, cm1 = M->cm1, inv_alpha = M->inv_alpha;
    for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t id = sids[p];
        double ph, r;
        if (phi_src) {
            ph = phi_src[id];
            r = r_src[id];
        } else {
            const U64x4 x = draw(id, seed);
            ph = phi_from_u53(x.x0 >> 11);
            r = radius_approx(x.x1 >> 11, R, cm1, inv_alpha);
        }
        float2 a;
        float4 q;
        filter_values(ph, r, G, etab, &a, &q);
        P.akey[p] = static_cast<uint32_t>(keys[p]);
        P.ang[p] = a;
        P.pms[p] = q;
        P.id[p] = id;
    }
}

__global__ void __launch_bounds__(256) gather_fp64_kernel(const Meta *M, uint64_t n, uint64_t seed,
                                                          const uint64_t *keys, const uint32_t *sids,
                                                          const double *phi_src, const double *r_by_id,
                                                          SortedPoints P)
{
    if (M->error || M->filter) return;
    for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t id = sids[p];
        const double ph = phi_src ? phi_src[id] : phi_from_u53(draw(id, seed).x0 >> 11);
        const double r = r_by_id[id];
        P.phi[p] = ph;
        P.r[p] = r;
        P.ch[p] = dm::cosh(r);
        P.sh[p] = dm::sinh(r);
        P.akey[p] = static_cast<uint32_t>(keys[p]);
        P.id[p] = id;
    }
}

// Batch gathers: CTA per tile; ids are local, the FP64 radius is by position.
__global__ void __launch_bounds__(256) gather_filter_batch_kernel(const Meta *metas, BatchTables bt,
                                                                  const uint64_t *keys, const uint32_t *sids,
                                                                  SortedPoints P)
{
    __shared__ float etab[2 * kExpTab + 1];
    const uint4 T = bt.tiles[blockIdx.x];
    const Meta *M = metas + T.x;
    for (int j = threadIdx.x; j <= 2 * kExpTab; j += blockDim.x) etab[j] = M->etab[j];
    __syncthreads();
    if (M->error || !M->filter) return;
    const double G = M->G, R = M->R, cm1 = M->cm1, inv_alpha = M->inv_alpha;
    const uint64_t seed = M->seed;
    for (uint32_t j = threadIdx.x; j < T.z; j += blockDim.x) {
        const uint32_t p = T.y + j;
        const uint32_t id = sids[p];
        const U64x4 x = draw(id, seed);
        const double ph = phi_from_u53(x.x0 >> 11);
        const double r = radius_approx(x.x1 >> 11, R, cm1, inv_alpha);
        float2 a;
        float4 q;
        filter_values(ph, r, G, etab, &a, &q);
        P.akey[p] = static_cast<uint32_t>(keys[p]);
        P.ang[p] = a;
        P.pms[p] = q;
        P.id[p] = id;
    }
}

__global__ void __launch_bounds__(256) gather_fp64_batch_kernel(const Meta *metas, BatchTables bt,
                                                                const uint64_t *keys, const uint32_t *sids,
                                                                const double *r_by_pos, SortedPoints P)
{
    const uint4 T = bt.tiles[blockIdx.x];
    const Meta *M = metas + T.x;
    if (M->error || M->filter) return;
    const uint64_t seed = M->seed;
    const uint32_t pos0 = bt.pt_off[T.x];
    for (uint32_t j = threadIdx.x; j < T.z; j += blockDim.x) {
        const uint32_t p = T.y + j;
        const uint32_t id = sids[p];
        const double ph = phi_from_u53(draw(id, seed).x0 >> 11);
        const double r = r_by_pos[pos0 + id];
        P.phi[p] = ph;
        P.r[p] = r;
        P.ch[p] = dm::cosh(r);
        P.sh[p] = dm::sinh(r);
        P.akey[p] = static_cast<uint32_t>(keys[p]);
        P.id[p] = id;
    }
}

// Per-graph results of a batch: {m low, m high, R low, R high} and {B, error}.
__global__ void batch_results_kernel(const Meta *metas, uint32_t G, uint4 *out)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const Meta *M = metas + g;
    const uint64_t m = M->m;
    const uint64_t Rb = static_cast<uint64_t>(__double_as_longlong(M->R));
    out[2 * g] = make_uint4(static_cast<uint32_t>(m), static_cast<uint32_t>(m >> 32), static_cast<uint32_t>(Rb),
                            static_cast<uint32_t>(Rb >> 32));
    out[2 * g + 1] = make_uint4(M->B, M->error, M->filter, 0u);
}

__global__ void points_by_id_kernel(const Meta *M, uint64_t n, uint64_t seed, double *phi, double *r)
{
    const double R = M->R, cm1 = M->cm1, inv_alpha = M->inv_alpha;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const U64x4 x = draw(i, seed);
        phi[i] = phi_from_u53(x.x0 >> 11);
        r[i] = radius_from_u53(x.x1 >> 11, R, cm1, inv_alpha);
    }
}

__global__ void dm_eval_kernel(int fn, const double *in, double *out, uint64_t count)
{
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const double x = in[i];
        double y;
        switch (fn) {
            case 0: y = dm::exp(x); break;
            case 1: y = dm::log(x); break;
            case 2: y = dm::cos(x); break;
            case 3: y = dm::cosh(x); break;
            case 4: y = dm::sinh(x); break;
            default: y = dm::asinh(x); break;
        }
        out[i] = y;
    }
}

unsigned grid_for(uint64_t n, int threads, int per_sm)
{
    const uint64_t need = ceil_div(n ? n : 1, static_cast<uint64_t>(threads));
    const uint64_t cap = static_cast<uint64_t>(num_sms()) * per_sm;
    return static_cast<unsigned>(need < cap ? need : cap);
}

}  // namespace

Status launch_plan(Meta *d_meta, const PlanArgs &a, cudaStream_t stream)
{
    Status st;
    plan_kernel<<<1, kPlanThreads, 0, stream>>>(d_meta, a);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_sample(Meta *d_meta, uint64_t n, uint64_t seed, uint64_t *keys, uint32_t *ids,
                     double *r_by_id, cudaStream_t stream)
{
    Status st;
    sample_kernel<<<grid_for(n, kSampleThreads, 8), kSampleThreads, 0, stream>>>(d_meta, n, seed, keys,
                                                                                ids, r_by_id);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_load_points(Meta *d_meta, uint64_t n, const double *phi, const double *r,
                          uint64_t *keys, uint32_t *ids, cudaStream_t stream)
{
    Status st;
    load_points_kernel<<<grid_for(n, kSampleThreads, 8), kSampleThreads, 0, stream>>>(d_meta, n, phi, r,
                                                                                     keys, ids);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_band_offsets(Meta *d_meta, cudaStream_t stream)
{
    Status st;
    band_offsets_kernel<<<1, 32, 0, stream>>>(d_meta);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_gather(const Meta *d_meta, uint64_t n, uint64_t seed, const uint64_t *sorted_keys,
                     const uint32_t *sorted_ids, const double *phi_src, const double *r_src,
                     const double *r64_src, SortedPoints P, cudaStream_t stream)
{
    Status st;
    gather_filter_kernel<<<grid_for(n, 256, 8), 256, 0, stream>>>(d_meta, n, seed, sorted_keys, sorted_ids,
                                                                phi_src, r_src, P);
    RHG_LAUNCH_CHECK();
    gather_fp64_kernel<<<grid_for(n, 256, 8), 256, 0, stream>>>(d_meta, n, seed, sorted_keys, sorted_ids,
                                                              phi_src, r64_src, P);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_plan_batch(Meta *metas, const PlanArgs *d_args, uint32_t G, cudaStream_t stream)
{
    Status st;
    plan_batch_kernel<<<G + 1, kPlanThreads, 0, stream>>>(metas, d_args, G);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_sample_batch(Meta *metas, const BatchTables &bt, uint64_t *keys, uint32_t *ids, double *r_by_pos,
                           cudaStream_t stream)
{
    Status st;
    if (!bt.num_tiles) return st;
    sample_batch_kernel<<<bt.num_tiles, kSampleThreads, 0, stream>>>(metas, bt, keys, ids, r_by_pos);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_band_offsets_batch(Meta *metas, const BatchTables &bt, cudaStream_t stream)
{
    Status st;
    band_offsets_batch_kernel<<<static_cast<unsigned>(ceil_div(bt.G, 128u)), 128, 0, stream>>>(metas, bt);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_gather_batch(const Meta *metas, const BatchTables &bt, const uint64_t *sorted_keys,
                           const uint32_t *sorted_ids, const double *r_by_pos, SortedPoints P, cudaStream_t stream)
{
    Status st;
    if (!bt.num_tiles) return st;
    gather_filter_batch_kernel<<<bt.num_tiles, 256, 0, stream>>>(metas, bt, sorted_keys, sorted_ids, P);
    RHG_LAUNCH_CHECK();
    gather_fp64_batch_kernel<<<bt.num_tiles, 256, 0, stream>>>(metas, bt, sorted_keys, sorted_ids, r_by_pos, P);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_batch_results(const Meta *metas, uint32_t G, uint4 *d_out, cudaStream_t stream)
{
    Status st;
    batch_results_kernel<<<static_cast<unsigned>(ceil_div(G, 128u)), 128, 0, stream>>>(metas, G, d_out);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_dm_eval(int fn, const double *in, double *out, uint64_t count, cudaStream_t stream)
{
    Status st;
    dm_eval_kernel<<<grid_for(count, 256, 8), 256, 0, stream>>>(fn, in, out, count);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_points_by_id(const Meta *d_meta, uint64_t n, uint64_t seed, double *phi, double *r,
                           cudaStream_t stream)
{
    Status st;
    points_by_id_kernel<<<grid_for(n, 256, 8), 256, 0, stream>>>(d_meta, n, seed, phi, r);
    RHG_LAUNCH_CHECK();
    return st;
}

}  // namespace rhg
