// query.cu -- the range query of Alg. 1 (the loop that dominates the running time,
// Sec. III-B): for each point v and each band b_i from v's own band outward,
// the getMinMaxPhi window, a binary search for the first and last candidate in
// the band's angle-sorted keys, and the FP64 distance test of every candidate;
// followed by the count / exclusive-scan / emit compaction of the edges, and the
// CSR assembly.
#include "kernels.h"

namespace rhg {
namespace {

constexpr int kQueryThreads = 128;

// Sec. III-B getMinMaxPhi: a neighbour w of v in band i (r_w >= c_i) satisfies
// cosh R >= cosh r_v cosh c_i - sinh r_v sinh c_i cos|phi_w - phi_v|, hence
// |phi_w - phi_v| <= theta with sin^2(theta/2) = (b - cosh(r_v - c_i)) /
// (2 sinh r_v sinh c_i), the same bound written without cancellation.  The
// threshold b is inflated so that the window also holds every pair the rounded
// FP64 predicate accepts: the predicate's rounding error is below
// 23 u cosh r_v cosh r_w and cosh r_w < cosh c_{i+1}, so b = (cosh R + 64 u
// cosh r_v cosh c_{i+1}) (1 + 1e-12) with u = 2^-53; the final relative and
// absolute margins cover the rounding of this evaluation.  Returns >= pi for the
// whole band.
__device__ __forceinline__ double window_theta(double rv, double chv, double shv, double coshR, double ci,
                                               double sinh_ci, double cosh_ci1)
{
    if (ci <= 0.0 || rv <= 0.0 || shv <= 0.0) return 4.0;
    constexpr double u = 0x1.0p-53;
    double b = coshR + 64.0 * u * chv * cosh_ci1;
    b = b * (1.0 + 1e-12);
    const double num = b - ::cosh(rv - ci);
    const double den = 2.0 * shv * sinh_ci;
    double Q = num / den;
    if (!(Q < 1.0)) return 4.0;
    if (Q < 0.0) Q = 0.0;
    return 2.0 * ::asin(::sqrt(Q)) * (1.0 + 1e-9) + 1e-12;
}

// first position in [lo, hi) whose key is >= x / > x
__device__ __forceinline__ uint64_t lower_bound_key(const uint32_t *a, uint64_t lo, uint64_t hi, uint32_t x)
{
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ uint64_t upper_bound_key(const uint32_t *a, uint64_t lo, uint64_t hi, uint32_t x)
{
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Candidate positions of the window [phi_v - theta, phi_v + theta] in band [s, e):
// up to two ranges (the window may wrap around 0 / 2 pi).
struct Ranges {
    uint64_t lo[2], hi[2];
    int count;
};

__device__ __forceinline__ Ranges window_ranges(const uint32_t *akey, uint64_t s, uint64_t e, double phv,
                                                double theta)
{
    Ranges R;
    if (theta >= dm::kPi) {
        R.lo[0] = s;
        R.hi[0] = e;
        R.count = 1;
        return R;
    }
    const double plo = phv - theta, phi_hi = phv + theta;
    if (plo < 0.0 || phi_hi >= dm::kTwoPi) {
        const double a = plo < 0.0 ? plo + dm::kTwoPi : plo;
        const double b = phi_hi >= dm::kTwoPi ? phi_hi - dm::kTwoPi : phi_hi;
        const uint64_t first = lower_bound_key(akey, s, e, angle_key(a));  // [first, e)
        const uint64_t last = upper_bound_key(akey, s, e, angle_key(b));   // [s, last)
        if (last > first) {  // the two pieces meet: the window covers the band
            R.lo[0] = s;
            R.hi[0] = e;
            R.count = 1;
        } else {
            R.lo[0] = first;
            R.hi[0] = e;
            R.lo[1] = s;
            R.hi[1] = last;
            R.count = 2;
        }
        return R;
    }
    R.lo[0] = lower_bound_key(akey, s, e, angle_key(plo));
    R.hi[0] = upper_bound_key(akey, s, e, angle_key(phi_hi));
    R.count = 1;
    return R;
}

struct QueryShared {
    double c[kMaxBands + 1];
    double cosh_c[kMaxBands + 1];
    double sinh_c[kMaxBands + 1];
    uint64_t start[kMaxBands + 1];
};

__device__ __forceinline__ void load_shared(QueryShared &S, const Meta *M)
{
    for (int j = threadIdx.x; j <= kMaxBands; j += blockDim.x) {
        S.c[j] = M->c[j];
        S.cosh_c[j] = M->cosh_c[j];
        S.sinh_c[j] = M->sinh_c[j];
        S.start[j] = M->band_start[j];
    }
}

// One thread per sorted position p; kMode 0 = count, 1 = pairs, 2 = directed CSR keys.
template <int kMode>
__global__ void __launch_bounds__(kQueryThreads) query_kernel(Meta *M, SortedPoints P, uint32_t *counts,
                                                              const uint64_t *offsets, uint32_t *pairs,
                                                              uint64_t *csr_keys)
{
    __shared__ QueryShared S;
    if (M->error) return;
    load_shared(S, M);
    const uint32_t B = M->B;
    const double coshR = M->coshR;
    __syncthreads();
    uint64_t cand_total = 0, near_total = 0;
    for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < P.n;
         p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t bv = static_cast<uint32_t>(P.key[p] >> 32);
        const double phv = P.phi[p], rv = P.r[p], chv = P.ch[p], shv = P.sh[p];
        const uint32_t idv = P.id[p];
        uint64_t out = kMode ? offsets[p] : 0;
        uint32_t cnt = 0;
        for (uint32_t i = bv; i < B; ++i) {
            const uint64_t s = S.start[i], e = S.start[i + 1];
            if (s == e) continue;
            const double theta = window_theta(rv, chv, shv, coshR, S.c[i], S.sinh_c[i], S.cosh_c[i + 1]);
            const Ranges rg = window_ranges(P.akey, s, e, phv, theta);
            for (int k = 0; k < rg.count; ++k) {
                uint64_t q = rg.lo[k];
                // same band: report the pair from the endpoint at the smaller position
                if (i == bv && q <= p) q = p + 1;
                for (; q < rg.hi[k]; ++q) {
                    const double L = predicate_L(phv, chv, shv, P.phi[q], P.ch[q], P.sh[q]);
                    if (kMode == 0) {
                        ++cand_total;
                        if (fabs(L - coshR) <= 1e-12 * coshR) ++near_total;
                    }
                    if (L <= coshR) {
                        if (kMode == 1) {
                            const uint32_t idw = P.id[q];
                            pairs[2 * out] = idv < idw ? idv : idw;
                            pairs[2 * out + 1] = idv < idw ? idw : idv;
                        } else if (kMode == 2) {
                            const uint64_t idw = P.id[q];
                            csr_keys[2 * out] = (static_cast<uint64_t>(idv) << 32) | idw;
                            csr_keys[2 * out + 1] = (idw << 32) | idv;
                        }
                        ++out;
                        ++cnt;
                    }
                }
            }
        }
        if (kMode == 0) counts[p] = cnt;
    }
    if (kMode == 0) {
        // warp-reduce the diagnostics before one atomic per warp
        for (int off = 16; off; off >>= 1) {
            cand_total += __shfl_down_sync(0xffffffffu, cand_total, off);
            near_total += __shfl_down_sync(0xffffffffu, near_total, off);
        }
        if ((threadIdx.x & 31) == 0) {
            if (cand_total) atomicAdd(reinterpret_cast<unsigned long long *>(&M->candidates), cand_total);
            if (near_total) atomicAdd(reinterpret_cast<unsigned long long *>(&M->near_threshold), near_total);
        }
    }
}

// ---------------------------------------------------------------- exclusive scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *total)
{
    __shared__ uint64_t warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    const uint64_t warp_prefix = warp ? warp_sums[warp - 1] : 0;
    *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *in, uint64_t n,
                                                                   uint64_t *block_sums)
{
    const uint64_t base = blockIdx.x * static_cast<uint64_t>(kScanChunk);
    uint64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t idx = base + static_cast<uint64_t>(i) * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    uint64_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint64_t *block_sums, uint64_t nb,
                                                                 uint64_t *total_dst)
{
    uint64_t carry = 0;
    for (uint64_t b = 0; b < nb; b += kScanThreads) {
        const uint64_t idx = b + threadIdx.x;
        const uint64_t v = idx < nb ? block_sums[idx] : 0;
        uint64_t tot;
        const uint64_t ex = block_exclusive_scan(v, &tot);
        if (idx < nb) block_sums[idx] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_dst = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t *in, uint64_t n,
                                                                  const uint64_t *block_offsets,
                                                                  uint64_t *out)
{
    // blocked arrangement: thread t owns kScanItems consecutive elements
    const uint64_t base = blockIdx.x * static_cast<uint64_t>(kScanChunk) +
                          static_cast<uint64_t>(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        s += v[i];
    }
    uint64_t total;
    uint64_t run = block_offsets[blockIdx.x] + block_exclusive_scan(s, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = run;
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

unsigned query_grid(uint64_t n)
{
    const uint64_t need = ceil_div(n ? n : 1, kQueryThreads);
    const uint64_t cap = static_cast<uint64_t>(num_sms()) * 16;
    return static_cast<unsigned>(need < cap ? need : cap);
}

}  // namespace

size_t scan_temp_bytes(uint64_t n) { return (ceil_div(n ? n : 1, kScanChunk) + 1) * sizeof(uint64_t); }

Status exclusive_scan_u32(const uint32_t *counts, uint64_t *offsets, uint64_t n, uint64_t *total_dst,
                          void *temp, cudaStream_t stream)
{
    Status st;
    const uint64_t nb = ceil_div(n ? n : 1, kScanChunk);
    uint64_t *sums = static_cast<uint64_t *>(temp);
    scan_reduce_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, stream>>>(counts, n, sums);
    RHG_LAUNCH_CHECK();
    scan_sums_kernel<<<1, kScanThreads, 0, stream>>>(sums, nb, total_dst);
    RHG_LAUNCH_CHECK();
    scan_apply_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, stream>>>(counts, n, sums, offsets);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_query_count(Meta *d_meta, SortedPoints P, uint32_t *counts, cudaStream_t stream)
{
    Status st;
    query_kernel<0><<<query_grid(P.n), kQueryThreads, 0, stream>>>(d_meta, P, counts, nullptr, nullptr,
                                                                   nullptr);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_query_emit(Meta *d_meta, SortedPoints P, const uint64_t *offsets, uint32_t *pairs,
                         uint64_t *csr_keys, cudaStream_t stream)
{
    Status st;
    if (csr_keys)
        query_kernel<2><<<query_grid(P.n), kQueryThreads, 0, stream>>>(d_meta, P, nullptr, offsets, nullptr,
                                                                       csr_keys);
    else
        query_kernel<1><<<query_grid(P.n), kQueryThreads, 0, stream>>>(d_meta, P, nullptr, offsets, pairs,
                                                                       nullptr);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_csr_finish(const uint64_t *sorted_keys, uint64_t entries, uint64_t n, uint64_t *row_ptr,
                         uint32_t *col, cudaStream_t stream)
{
    Status st;
    if (entries == 0) {
        fill_u64_kernel<<<static_cast<unsigned>(ceil_div(n + 1, 256) < 4096 ? ceil_div(n + 1, 256) : 4096), 256,
                          0, stream>>>(row_ptr, n + 1, 0);
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
