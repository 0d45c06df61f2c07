// sort.cu -- stable LSD radix sort of 64-bit keys with optional uint32 payload
// (Alg. 1, angular sort within each band: one global sort keyed by (band, angle
// key) orders every band at once).
//
// One pass per 8-bit digit:
//   upsweep   each CTA histograms the digit over its contiguous chunk;
//   scan      one CTA per digit turns its row of the digit-major [digit][cta]
//             counts into an exclusive prefix and a digit total (the downsweep
//             adds the exclusive scan of the totals);
//   downsweep each CTA walks its chunk tile by tile; inside a tile every warp
//             ranks its 32 x kItems keys with __match_any_sync, warps are combined
//             by a per-digit prefix over warps, so the order of equal digits is the
//             input order (stable); the tile is staged in shared memory in digit
//             order and written out from there, one contiguous run per digit.
#include "kernels.h"
#include "stages.cuh"

namespace rhg {
namespace {

using namespace stg;

struct Grid {
    uint32_t ctas;
    uint64_t tiles_per_cta;
};

Grid sort_grid(uint64_t n)
{
    const uint64_t tiles = ceil_div(n ? n : 1, kTile);
    const uint64_t max_ctas = static_cast<uint64_t>(num_sms()) * 4;
    const uint64_t ctas = tiles < max_ctas ? tiles : max_ctas;
    return Grid{static_cast<uint32_t>(ctas), ceil_div(tiles, ctas)};
}

__global__ void __launch_bounds__(kThreads) upsweep_kernel(const uint64_t *keys, uint64_t n, int shift,
                                                           uint64_t tiles_per_cta, uint32_t *counts)
{
    __shared__ uint32_t hist[kRadix];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t begin = blockIdx.x * tiles_per_cta * kTile;
    uint64_t end = begin + tiles_per_cta * kTile;
    if (end > n) end = n;
    for (uint64_t i = begin + threadIdx.x; i < end; i += kThreads)
        atomicAdd(&hist[(keys[i] >> shift) & (kRadix - 1)], 1u);
    __syncthreads();
    counts[static_cast<uint64_t>(threadIdx.x) * gridDim.x + blockIdx.x] = hist[threadIdx.x];
}

// Row d of the digit-major counts (the CTAs' counts of digit d) becomes its
// exclusive prefix, in place, and totals[d] its sum; one CTA per digit.
__global__ void __launch_bounds__(kThreads) scan_rows_kernel(uint32_t *counts, uint32_t ctas, uint32_t *totals)
{
    __shared__ uint32_t warp_sum[kWarps];
    uint32_t *row = counts + static_cast<uint64_t>(blockIdx.x) * ctas;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < ctas; base += kThreads) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < ctas ? row[i] : 0u;
        uint32_t incl = v;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        uint32_t before = carry;
        for (int w = 0; w < warp; ++w) before += warp_sum[w];
        uint32_t chunk = 0;
        for (int w = 0; w < kWarps; ++w) chunk += warp_sum[w];
        if (i < ctas) row[i] = before + incl - v;
        carry += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

template <bool kValues>
__global__ void __launch_bounds__(kThreads) downsweep_kernel(const uint64_t *keys_in, uint64_t *keys_out,
                                                             const uint32_t *vals_in, uint32_t *vals_out,
                                                             uint64_t n, int shift, uint64_t tiles_per_cta,
                                                             const uint32_t *offsets, const uint32_t *totals)
{
    __shared__ TileSmem sm;
    __shared__ uint32_t sval[kValues ? kTile : 1];
    // this CTA's first position of digit d: keys of smaller digits (exclusive
    // scan of the digit totals) plus keys of digit d in earlier CTAs
    sm.digit_base[threadIdx.x] = block_exclusive(totals[threadIdx.x], sm.warp_sum) +
                                 offsets[static_cast<uint64_t>(threadIdx.x) * gridDim.x + blockIdx.x];
    __syncthreads();
    const uint64_t chunk = blockIdx.x * tiles_per_cta * kTile;
    for (uint64_t t = 0; t < tiles_per_cta; ++t) {
        const uint64_t tile = chunk + t * kTile;
        if (tile >= n) break;
        const uint32_t cnt = n - tile < static_cast<uint64_t>(kTile) ? static_cast<uint32_t>(n - tile) : kTile;
        tile_pass<kValues>(keys_in, keys_out, vals_in, vals_out, tile, cnt, shift, sm, sval);
    }
}

}  // namespace

size_t radix_temp_bytes(uint64_t n)
{
    const Grid g = sort_grid(n);
    return static_cast<size_t>(kRadix) * (g.ctas + 1) * sizeof(uint32_t);
}

Status radix_sort(uint64_t n, uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt,
                  const int *shifts, int num_shifts, void *temp, uint64_t **keys_out,
                  uint32_t **vals_out, cudaStream_t stream)
{
    Status st;
    uint64_t *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    if (n > 1) {
        const Grid g = sort_grid(n);
        uint32_t *counts = static_cast<uint32_t *>(temp);
        uint32_t *totals = counts + static_cast<size_t>(kRadix) * g.ctas;
        for (int s = 0; s < num_shifts; ++s) {
            upsweep_kernel<<<g.ctas, kThreads, 0, stream>>>(kin, n, shifts[s], g.tiles_per_cta, counts);
            RHG_LAUNCH_CHECK();
            scan_rows_kernel<<<kRadix, kThreads, 0, stream>>>(counts, g.ctas, totals);
            RHG_LAUNCH_CHECK();
            if (vals) {
                downsweep_kernel<true><<<g.ctas, kThreads, 0, stream>>>(kin, kout, vin, vout, n, shifts[s],
                                                                       g.tiles_per_cta, counts, totals);
            } else {
                downsweep_kernel<false><<<g.ctas, kThreads, 0, stream>>>(kin, kout, nullptr, nullptr, n,
                                                                        shifts[s], g.tiles_per_cta, counts, totals);
            }
            RHG_LAUNCH_CHECK();
            uint64_t *tk = kin;
            kin = kout;
            kout = tk;
            uint32_t *tv = vin;
            vin = vout;
            vout = tv;
        }
    }
    *keys_out = kin;
    if (vals_out) *vals_out = vin;
    return st;
}

}  // namespace rhg
