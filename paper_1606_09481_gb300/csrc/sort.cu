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

namespace rhg {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // keys per tile
constexpr int kRadix = 256;

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

// ---- segmented (batch): tiles of one graph each, per-tile digit counts
static_assert(kTile == static_cast<int>(kTilePoints), "batch tiles are sort tiles");

__global__ void __launch_bounds__(kThreads) seg_upsweep_kernel(const uint64_t *keys, BatchTables bt, int shift,
                                                               uint32_t *counts)
{
    __shared__ uint32_t hist[kRadix];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const uint4 T = bt.tiles[blockIdx.x];
    for (uint32_t j = threadIdx.x; j < T.z; j += kThreads) atomicAdd(&hist[(keys[T.y + j] >> shift) & (kRadix - 1)], 1u);
    __syncthreads();
    counts[static_cast<uint64_t>(blockIdx.x) * kRadix + threadIdx.x] = hist[threadIdx.x];
}

// CTA per graph: counts[t][d] of the graph's tiles become the output position of
// tile t's first key of digit d (graph start + keys of smaller digits + keys of
// digit d in earlier tiles of the graph).
__global__ void __launch_bounds__(kThreads) seg_scan_kernel(BatchTables bt, uint32_t *counts)
{
    __shared__ uint32_t warp_sum[kWarps];
    const uint32_t g = blockIdx.x, d = threadIdx.x;
    const uint32_t t0 = bt.tile_first[g], t1 = bt.tile_first[g + 1];
    uint32_t run = 0;
    for (uint32_t t = t0; t < t1; ++t) {
        uint32_t &c = counts[static_cast<uint64_t>(t) * kRadix + d];
        const uint32_t v = c;
        c = run;
        run += v;
    }
    const uint32_t base = bt.pt_off[g] + block_exclusive(run, warp_sum);
    for (uint32_t t = t0; t < t1; ++t) counts[static_cast<uint64_t>(t) * kRadix + d] += base;
}

template <bool kValues>
__global__ void __launch_bounds__(kThreads) seg_downsweep_kernel(const uint64_t *keys_in, uint64_t *keys_out,
                                                                 const uint32_t *vals_in, uint32_t *vals_out,
                                                                 BatchTables bt, int shift, const uint32_t *offsets)
{
    __shared__ TileSmem sm;
    __shared__ uint32_t sval[kValues ? kTile : 1];
    const uint4 T = bt.tiles[blockIdx.x];
    sm.digit_base[threadIdx.x] = offsets[static_cast<uint64_t>(blockIdx.x) * kRadix + threadIdx.x];
    __syncthreads();
    tile_pass<kValues>(keys_in, keys_out, vals_in, vals_out, T.y, T.z, shift, sm, sval);
}

}  // namespace

size_t radix_temp_bytes(uint64_t n)
{
    const Grid g = sort_grid(n);
    return static_cast<size_t>(kRadix) * (g.ctas + 1) * sizeof(uint32_t);
}

size_t segmented_temp_bytes(uint32_t num_tiles) { return static_cast<size_t>(kRadix) * (num_tiles + 1) * 4; }

Status segmented_radix_sort(const BatchTables &bt, uint64_t *keys, uint64_t *keys_alt, uint32_t *vals,
                            uint32_t *vals_alt, const int *shifts, int num_shifts, void *temp, uint64_t **keys_out,
                            uint32_t **vals_out, cudaStream_t stream)
{
    Status st;
    uint64_t *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    if (bt.num_tiles && bt.G) {
        uint32_t *counts = static_cast<uint32_t *>(temp);
        for (int s = 0; s < num_shifts; ++s) {
            seg_upsweep_kernel<<<bt.num_tiles, kThreads, 0, stream>>>(kin, bt, shifts[s], counts);
            RHG_LAUNCH_CHECK();
            seg_scan_kernel<<<bt.G, kThreads, 0, stream>>>(bt, counts);
            RHG_LAUNCH_CHECK();
            if (vals) {
                seg_downsweep_kernel<true><<<bt.num_tiles, kThreads, 0, stream>>>(kin, kout, vin, vout, bt, shifts[s],
                                                                                 counts);
            } else {
                seg_downsweep_kernel<false><<<bt.num_tiles, kThreads, 0, stream>>>(kin, kout, nullptr, nullptr, bt,
                                                                                  shifts[s], counts);
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
