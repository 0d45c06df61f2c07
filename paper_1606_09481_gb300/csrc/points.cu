// points.cu -- the point pipeline: disk radius R (Sec. III-B getTargetRadius),
// band boundaries (Sec. III-A), Philox sampling of (phi, r) by inverse CDF
// (Alg. 1 sampling step, Eq. 1), band assignment (Alg. 1 band insertion)
// and the gather of the (band, angle)-sorted structure-of-arrays.
#include "kernels.h"
#include "stages.cuh"

namespace rhg {
namespace {

using namespace stg;

__global__ void __launch_bounds__(kPlanThreads) plan_kernel(Meta *M, PlanArgs a)
{
    __shared__ PlanSmem PS;
    plan_block(M, a, 8, PS);
}

// Points by id: sort key (band << 32 | angle key) and id.  In filter mode the band
// comes from the radial variate compared with the band thresholds (band_of_u53, no
// FP64); otherwise from the FP64 radius, which is also stored by id for the gather.
// With bucket_counts, every point also counts in its sort bucket (bucket sort).
__global__ void __launch_bounds__(kSampleThreads) sample_kernel(Meta *M, uint64_t n, uint64_t seed,
                                                                uint64_t *keys, uint32_t *ids,
                                                                double *r_by_id, uint32_t *bucket_counts)
{
    __shared__ double c[kMaxBands + 1];
    __shared__ uint64_t bu[kMaxBands + 1];
    __shared__ uint32_t bk_off[kMaxBands + 1], bk_bits[kMaxBands];
    __shared__ unsigned int hist[kMaxBands];
    const uint32_t B = M->B;
    const bool filter = M->filter != 0;
    const double R = M->R, cm1 = M->cm1, inv_alpha = M->inv_alpha;
    if (threadIdx.x <= B) {
        c[threadIdx.x] = M->c[threadIdx.x];
        bu[threadIdx.x] = M->band_u[threadIdx.x];
        bk_off[threadIdx.x] = M->bk_off[threadIdx.x];
        if (threadIdx.x < B) bk_bits[threadIdx.x] = M->bk_bits[threadIdx.x];
    }
    if (threadIdx.x < kMaxBands) hist[threadIdx.x] = 0;
    __syncthreads();
    if (M->error) return;
    // warp-uniform trip count (the histogram is counted per warp)
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i0 = blockIdx.x * static_cast<uint64_t>(blockDim.x) + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
        const uint64_t i = i0 + (threadIdx.x & 31u);
        uint32_t b = kMaxBands, akey = 0;
        if (i < n) {
            const U64x4 x = draw(i, seed);
            akey = static_cast<uint32_t>(x.x0 >> 32);
            if (filter) {
                b = band_of_u53(x.x1 >> 11, bu, B);
            } else {
                const double r = radius_from_u53(x.x1 >> 11, R, cm1, inv_alpha);
                r_by_id[i] = r;
                b = band_of(r, c, B);
            }
            keys[i] = (static_cast<uint64_t>(b) << 32) | akey;
            if (ids) ids[i] = static_cast<uint32_t>(i);
        }
        hist_add_warp(hist, b);
        if (bucket_counts) {  // one global atomic per distinct bucket among the lanes
            const uint32_t bk = b < B ? bucket_of((static_cast<uint64_t>(b) << 32) | akey, bk_off, bk_bits)
                                      : 0xffffffffu;
            const unsigned peers = __match_any_sync(0xffffffffu, bk);
            if (bk != 0xffffffffu && (peers & ((1u << (threadIdx.x & 31u)) - 1u)) == 0)
                atomicAdd(&bucket_counts[bk], static_cast<uint32_t>(__popc(peers)));
        }
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

__global__ void band_offsets_kernel(Meta *M)
{
    if (threadIdx.x == 0) band_offsets_one(M, 0, 0);
}

__global__ void __launch_bounds__(256) gather_filter_kernel(const Meta *M, uint64_t n, uint64_t seed,
                                                            const uint64_t *keys, const uint32_t *sids,
                                                            const double *phi_src, const double *r_src,
                                                            SortedPoints P)
{
    __shared__ float etab[2 * kExpTab + 1];
    __shared__ YTab Y;
    for (int j = threadIdx.x; j <= 2 * kExpTab; j += blockDim.x) etab[j] = M->etab[j];
    load_ytab(Y, M);
    __syncthreads();
    if (M->error || !M->filter) return;
    const double G = M->G;
    for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t id = sids[p];
        float2 a;
        float4 q;
        if (phi_src) {  // caller's points: from the FP64 coordinates
            filter_values(phi_src[id], r_src[id], G, etab, &a, &q);
        } else {        // generated points: from the variates, without FP64
            const U64x4 x = draw(id, seed);
            filter_values_u53(x.x0 >> 11, x.x1 >> 11, yref(Y), &a, &q);
        }
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
                     double *r_by_id, uint32_t *bucket_counts, cudaStream_t stream)
{
    Status st;
    sample_kernel<<<grid_for(n, kSampleThreads, 8), kSampleThreads, 0, stream>>>(d_meta, n, seed, keys,
                                                                                ids, r_by_id, bucket_counts);
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
