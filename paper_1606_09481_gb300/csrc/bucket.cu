// bucket.cu -- bucket sort of generated points by (band, angle key, id) (Alg. 1,
// angular sort within each band) with the gather of the sorted point arrays
// fused into its last pass.
//
// The angles of generated points are uniform, so a band's points spread evenly
// over buckets cut by the top bits of the angle key (Meta::bk_off / bk_bits, set
// by the plan from the band's expected count).  Passes:
//   count    points per bucket (the sampler counts them; bucket_count_kernel for
//            caller keys);
//   scan     bucket starts = exclusive scan of the counts (one CTA, which also
//            sets the band offsets);
//   scatter  (angle key << 32 | id) to its bucket, at a cursor taken with an
//            atomic add (the order inside a bucket is arbitrary here);
//   sort     one CTA per bucket: the bucket into shared memory, a counting pass
//            on the next 8 bits of the angle key, then every sub-bucket (a few
//            points) sorted by one thread, so that the bucket is in (angle key,
//            id) order; then each position is handed on (gather or output).  A
//            bucket above kBucketCap points, or with a sub-bucket above kSubMax,
//            takes an LSD radix sort of its range in global memory instead
//            (never for uniform angles at these bucket sizes, but any input sorts).
#include "kernels.h"
#include "stages.cuh"

namespace rhg {
namespace {

constexpr int kBkThreads = stg::kThreads;

__global__ void __launch_bounds__(kBkThreads) bucket_count_kernel(Meta *M, uint64_t n, const uint64_t *keys,
                                                                  uint32_t *counts)
{
    __shared__ uint32_t off[kMaxBands + 1], bits[kMaxBands];
    const uint32_t B = M->B;
    if (threadIdx.x <= B) {
        off[threadIdx.x] = M->bk_off[threadIdx.x];
        if (threadIdx.x < B) bits[threadIdx.x] = M->bk_bits[threadIdx.x];
    }
    __syncthreads();
    bool bad = false;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        const uint64_t k = keys[i];
        if ((k >> 32) >= B) {
            bad = true;
            continue;
        }
        atomicAdd(&counts[bucket_of(k, off, bits)], 1u);
    }
    if (bad) atomicMax(&M->error, kErrBadPoint);
}

// Band offsets (band_offsets_one) and the bucket starts; start[nb] = n.
__global__ void __launch_bounds__(1024) bucket_scan_kernel(Meta *M, uint32_t *counts, uint32_t *start)
{
    __shared__ uint32_t warp_sum[32];
    if (threadIdx.x == 0) stg::band_offsets_one(M, 0, 0);
    if (M->error) return;
    const uint32_t nb = M->nbuckets;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nb; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? counts[i] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        uint32_t before = carry, chunk = 0;
        for (int w = 0; w < 32; ++w) {
            const uint32_t ws = warp_sum[w];
            if (w < warp) before += ws;
            chunk += ws;
        }
        if (i < nb) {
            const uint32_t excl = before + incl - v;
            start[i] = excl;
            counts[i] = excl;  // the scatter's cursor
        }
        carry += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[nb] = carry;
}

__global__ void __launch_bounds__(kBkThreads) bucket_scatter_kernel(const Meta *M, uint64_t n, const uint64_t *keys,
                                                                    uint32_t *cursor, uint64_t *comp)
{
    __shared__ uint32_t off[kMaxBands + 1], bits[kMaxBands];
    const uint32_t B = M->B;
    if (threadIdx.x <= B) {
        off[threadIdx.x] = M->bk_off[threadIdx.x];
        if (threadIdx.x < B) bits[threadIdx.x] = M->bk_bits[threadIdx.x];
    }
    __syncthreads();
    if (M->error) return;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        const uint64_t k = keys[i];
        const uint32_t pos = atomicAdd(&cursor[bucket_of(k, off, bits)], 1u);
        comp[pos] = (k << 32) | static_cast<uint32_t>(i);
    }
}

// One CTA per bucket (grid-stride).  kGather: the sorted key goes back into comp
// and the point's filter values (filter mode: FP32/integer from its variates) or
// FP64 values go to P; else the sorted keys and ids go to out_keys / out_ids.
template <bool kGather>
__global__ void __launch_bounds__(kBkThreads, 4) bucket_sort_kernel(BucketArgs a)
{
    __shared__ stg::BucketSmem SB;
    __shared__ uint32_t off[kMaxBands + 1], bits[kMaxBands];
    __shared__ stg::YTab Y;
    Meta *M = a.M;
    const uint32_t B = M->B, nb = M->nbuckets;
    if (threadIdx.x <= B) {
        off[threadIdx.x] = M->bk_off[threadIdx.x];
        if (threadIdx.x < B) bits[threadIdx.x] = M->bk_bits[threadIdx.x];
    }
    if (kGather) stg::load_ytab(Y, M);
    __syncthreads();
    if (M->error) return;
    const bool filter = M->filter != 0;
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const uint32_t s = a.start[b], cnt = a.start[b + 1] - s;
        uint32_t band = 0;  // the largest j < B with off[j] <= b
        for (uint32_t step = 32; step; step >>= 1)
            if (band + step < B && off[band + step] <= b) band += step;
        const int rest = 32 - static_cast<int>(bits[band]);  // angle-key bits below the bucket's
        const int dsh = 32 + (rest > 8 ? rest - 8 : 0);     // the next 8 of them, in the composite
        const uint64_t *sorted = stg::sort_bucket(a.comp, a.scratch, s, cnt, dsh, SB);
        for (uint32_t k = threadIdx.x; k < cnt; k += kBkThreads) {
            const uint64_t c = sorted[k];
            const uint32_t p = s + k, id = static_cast<uint32_t>(c), akey = static_cast<uint32_t>(c >> 32);
            const uint64_t key = (static_cast<uint64_t>(band) << 32) | akey;
            if (kGather) {
                a.comp[p] = key;
                a.P.akey[p] = akey;
                a.P.id[p] = id;
                const U64x4 x = draw(id, a.seed);
                if (filter) {
                    float2 ang;
                    float4 pms;
                    stg::filter_values_u53(x.x0 >> 11, x.x1 >> 11, stg::yref(Y), &ang, &pms);
                    a.P.ang[p] = ang;
                    a.P.pms[p] = pms;
                } else {
                    const double r = a.r_by_id[id];
                    a.P.phi[p] = phi_from_u53(x.x0 >> 11);
                    a.P.r[p] = r;
                    a.P.ch[p] = dm::cosh(r);
                    a.P.sh[p] = dm::sinh(r);
                }
            } else {
                a.out_keys[p] = key;
                a.out_ids[p] = id;
            }
        }
    }
}

unsigned grid_cap(uint64_t n, int threads, int per_sm)
{
    const uint64_t need = (n ? n : 1) / threads + 1;
    const uint64_t cap = static_cast<uint64_t>(num_sms()) * per_sm;
    return static_cast<unsigned>(need < cap ? need : cap);
}

}  // namespace

Status launch_bucket_count(const BucketArgs &a, const uint64_t *keys, cudaStream_t stream)
{
    Status st;
    bucket_count_kernel<<<grid_cap(a.n, kBkThreads, 8), kBkThreads, 0, stream>>>(a.M, a.n, keys, a.counts);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_bucket_scan(const BucketArgs &a, cudaStream_t stream)
{
    Status st;
    bucket_scan_kernel<<<1, 1024, 0, stream>>>(a.M, a.counts, a.start);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_bucket_scatter(const BucketArgs &a, const uint64_t *keys, cudaStream_t stream)
{
    Status st;
    bucket_scatter_kernel<<<grid_cap(a.n, kBkThreads, 8), kBkThreads, 0, stream>>>(a.M, a.n, keys, a.counts,
                                                                                   a.comp);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_bucket_sort(const BucketArgs &a, bool gather, cudaStream_t stream)
{
    Status st;
    // one CTA per bucket, 4 resident per SM (registers)
    const uint64_t buckets = bucket_entries(a.n);
    const uint64_t cap = static_cast<uint64_t>(num_sms()) * 4;
    const unsigned grid = static_cast<unsigned>(buckets < cap ? buckets : cap);
    if (gather) bucket_sort_kernel<true><<<grid, kBkThreads, 0, stream>>>(a);
    else bucket_sort_kernel<false><<<grid, kBkThreads, 0, stream>>>(a);
    RHG_LAUNCH_CHECK();
    return st;
}

}  // namespace rhg
