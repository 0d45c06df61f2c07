// dynamic.cu -- the dynamic model (Sec. III-C): step values, one movement step
// (rotation and the radial movement of Algorithm 2 with reflection at 0 and R,
// in the coordinate cosh(alpha r) - 1 under which Theorem 1 holds)
// and the pieces of an edge-list update after a step: marking the moved
// vertices, listing their sorted positions, a scan of per-vertex counts, and
// keeping the old edges whose endpoints both stayed.
#include "kernels.h"

namespace rhg {
namespace {

using dm::add;
using dm::mul;
using dm::sub;

constexpr int kThreads = 256;
constexpr double kBelowTwoPi = 0x1.921fb54442d17p+2;  // largest double below 2 pi

unsigned grid(uint64_t work, int per_sm = 8)
{
    const uint64_t need = ceil_div(work ? work : 1, kThreads);
    const uint64_t cap = static_cast<uint64_t>(num_sms()) * per_sm;
    return static_cast<unsigned>(need < cap ? need : cap);
}

// Step values of vertex i from Philox counter (i, 1, 0, 0), key (seed, 0):
// tau = lo + (hi - lo) U with U = (word >> 11) 2^-53 (words 0 and 1).
__global__ void draw_movement_kernel(uint64_t n, uint64_t seed, double phi_lo, double phi_w, double r_lo, double r_w,
                                     double *tau_phi, double *tau_r)
{
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const U64x4 x = philox4x64_10(U64x4{i, 1, 0, 0}, seed, 0);
        const double u0 = static_cast<double>(x.x0 >> 11) * kU53;
        const double u1 = static_cast<double>(x.x1 >> 11) * kU53;
        tau_phi[i] = add(phi_lo, mul(phi_w, u0));
        tau_r[i] = add(r_lo, mul(r_w, u1));
    }
}

// One movement step of the listed vertices, in place.  Rotation: phi + tau_phi
// brought into [0, 2 pi).  Radial (Algorithm 2 in the coordinate that Theorem 1
// needs, the one that is uniform under Eq. 1): x = cosh(alpha r) - 1, evaluated
// as 2 sinh^2(alpha r / 2); y = x + tau_r, mirrored at top = cosh(alpha R) - 1 or
// 0 while outside (tau_r changes sign each time); r = 2 asinh(sqrt(y / 2)) / alpha,
// at most R.  (Algorithm 2 prints sinh(alpha r), which is not uniform under
// Eq. 1, so a walk in it does not keep the density.)  Ids at or above n are
// skipped.
__global__ void move_kernel(const uint32_t *ids, uint64_t count, uint64_t n, double *phi, double *r,
                            const double *tau_phi, double *tau_r, double R, double alpha)
{
    const double top = sub(dm::cosh(mul(alpha, R)), 1.0);
    const double inv_alpha = dm::div(1.0, alpha);
    for (uint64_t j = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; j < count;
         j += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t i = ids[j];
        if (i >= n) continue;
        double p = add(phi[i], tau_phi[i]);
        for (int it = 0; it < 64 && p >= dm::kTwoPi; ++it) p = sub(p, dm::kTwoPi);
        for (int it = 0; it < 64 && p < 0.0; ++it) p = add(p, dm::kTwoPi);
        if (p >= dm::kTwoPi) p = kBelowTwoPi;
        if (p < 0.0) p = 0.0;
        double tr = tau_r[i];
        const double s = dm::sinh(mul(mul(alpha, r[i]), 0.5));
        double y = add(mul(mul(s, s), 2.0), tr);
        for (int it = 0; it < 64 && (y > top || y < 0.0); ++it) {
            y = y > top ? sub(add(top, top), y) : -y;
            tr = -tr;
        }
        if (y > top) y = top;
        if (y < 0.0) y = 0.0;
        double z = mul(mul(dm::asinh(__dsqrt_rn(mul(y, 0.5))), 2.0), inv_alpha);
        if (z > R) z = R;
        phi[i] = p;
        r[i] = z;
        tau_r[i] = tr;
    }
}

__global__ void fill_u8_kernel(uint8_t *a, uint64_t count, uint8_t v)
{
    for (uint64_t j = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; j < count;
         j += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        a[j] = v;
}

__global__ void mark_kernel(const uint32_t *ids, uint64_t count, uint64_t n, uint8_t *moved_by_id,
                            uint32_t *moved_bits)
{
    for (uint64_t j = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; j < count;
         j += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t i = ids[j];
        if (i < n) {
            moved_by_id[i] = 1;
            atomicOr(moved_bits + (i >> 5), 1u << (i & 31));
        }
    }
}

__global__ void fill_u32_kernel(uint32_t *a, uint64_t count)
{
    for (uint64_t j = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; j < count;
         j += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        a[j] = 0;
}

// Moved flag by sorted position, and the sorted positions of the moved vertices
// (one atomic per block; order within a block kept).
__global__ void __launch_bounds__(kThreads) owners_kernel(const Meta *M, const uint32_t *sorted_ids, uint64_t n,
                                                          const uint8_t *moved_by_id, uint8_t *moved_by_pos,
                                                          uint32_t *owners, uint64_t cap, unsigned long long *counter)
{
    if (M->error) return;  // an earlier stage failed: the sorted ids may be undefined
    __shared__ uint32_t warp_cnt[kThreads / 32];
    __shared__ unsigned long long block_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t base = static_cast<uint64_t>(blockIdx.x) * kThreads; base < n;
         base += static_cast<uint64_t>(gridDim.x) * kThreads) {
        const uint64_t p = base + threadIdx.x;
        const bool mv = p < n && moved_by_id[sorted_ids[p]] != 0;
        if (p < n) moved_by_pos[p] = mv ? 1 : 0;
        const uint32_t b = __ballot_sync(0xffffffffu, mv);
        if (lane == 0) warp_cnt[warp] = __popc(b);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += warp_cnt[w];
            block_base = t ? atomicAdd(counter, static_cast<unsigned long long>(t)) : 0ull;
        }
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += warp_cnt[w];
        const uint64_t at = block_base + before + __popc(b & ((1u << lane) - 1u));
        if (mv && at < cap) owners[at] = static_cast<uint32_t>(p);
        __syncthreads();
    }
}

// Exclusive scan of count uint32 values into uint64 offsets, total at out[count]:
// per-block sums, one CTA over the sums, then per-block scans with their base.
constexpr int kScanItems = 4;
constexpr int kScanBlock = kThreads * kScanItems;

__device__ __forceinline__ uint64_t block_scan_excl(uint64_t v, uint64_t *warp_sum, uint64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = v;
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    uint64_t before = 0, all = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
        if (w < warp) before += warp_sum[w];
        all += warp_sum[w];
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(kThreads) scan_sums_kernel(const uint32_t *in, uint64_t count, uint64_t *sums)
{
    __shared__ uint64_t ws[kThreads / 32];
    const uint64_t b0 = static_cast<uint64_t>(blockIdx.x) * kScanBlock;
    uint64_t v = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const uint64_t j = b0 + static_cast<uint64_t>(threadIdx.x) * kScanItems + k;
        if (j < count) v += in[j];
    }
    uint64_t total;
    block_scan_excl(v, ws, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads) scan_top_kernel(uint64_t *sums, uint64_t blocks)
{
    __shared__ uint64_t ws[kThreads / 32];
    uint64_t carry = 0;
    for (uint64_t b0 = 0; b0 < blocks; b0 += kThreads) {
        const uint64_t j = b0 + threadIdx.x;
        const uint64_t v = j < blocks ? sums[j] : 0;
        uint64_t total;
        const uint64_t ex = block_scan_excl(v, ws, &total);
        if (j < blocks) sums[j] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) sums[blocks] = carry;
}

__global__ void __launch_bounds__(kThreads) scan_apply_kernel(const uint32_t *in, uint64_t count, const uint64_t *sums,
                                                              uint64_t *out)
{
    __shared__ uint64_t ws[kThreads / 32];
    const uint64_t b0 = static_cast<uint64_t>(blockIdx.x) * kScanBlock;
    uint64_t v[kScanItems], s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const uint64_t j = b0 + static_cast<uint64_t>(threadIdx.x) * kScanItems + k;
        v[k] = j < count ? in[j] : 0;
        s += v[k];
    }
    uint64_t total;
    uint64_t run = sums[blockIdx.x] + block_scan_excl(s, ws, &total);
    for (int k = 0; k < kScanItems; ++k) {
        const uint64_t j = b0 + static_cast<uint64_t>(threadIdx.x) * kScanItems + k;
        if (j < count) out[j] = run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = sums[gridDim.x];
}

// The old edges whose endpoints both stayed (moved ids as a bitset), appended
// through the counter with one atomic per block and kKeepItems pairs per thread
// in flight; pairs past the capacity are counted but not written.
constexpr int kKeepItems = 4;

__global__ void __launch_bounds__(kThreads) keep_old_kernel(const uint2 *old_pairs, uint64_t m_old,
                                                            const uint32_t *moved_bits, uint64_t n, uint2 *out,
                                                            uint64_t cap, unsigned long long *counter)
{
    __shared__ uint32_t warp_cnt[kThreads / 32];
    __shared__ unsigned long long block_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint64_t kSpan = static_cast<uint64_t>(kThreads) * kKeepItems;
    for (uint64_t base = static_cast<uint64_t>(blockIdx.x) * kSpan; base < m_old;
         base += static_cast<uint64_t>(gridDim.x) * kSpan) {
        uint2 e[kKeepItems];
        bool keep[kKeepItems];
        uint32_t b[kKeepItems], mine = 0;
#pragma unroll
        for (int t = 0; t < kKeepItems; ++t) {  // pair base + t * kThreads + threadIdx.x (coalesced)
            const uint64_t j = base + static_cast<uint64_t>(t) * kThreads + threadIdx.x;
            e[t] = j < m_old ? old_pairs[j] : make_uint2(0xffffffffu, 0xffffffffu);
        }
#pragma unroll
        for (int t = 0; t < kKeepItems; ++t) {
            keep[t] = e[t].x < n && e[t].y < n && !((__ldg(moved_bits + (e[t].x >> 5)) >> (e[t].x & 31)) & 1u) &&
                      !((__ldg(moved_bits + (e[t].y >> 5)) >> (e[t].y & 31)) & 1u);
            b[t] = __ballot_sync(0xffffffffu, keep[t]);
            mine += __popc(b[t]);
        }
        if (lane == 0) warp_cnt[warp] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < kThreads / 32; ++w) tot += warp_cnt[w];
            block_base = tot ? atomicAdd(counter, static_cast<unsigned long long>(tot)) : 0ull;
        }
        __syncthreads();
        uint64_t at = block_base;
        for (int w = 0; w < warp; ++w) at += warp_cnt[w];
#pragma unroll
        for (int t = 0; t < kKeepItems; ++t) {
            const uint64_t pos = at + __popc(b[t] & ((1u << lane) - 1u));
            if (keep[t] && pos < cap) out[pos] = e[t];
            at += __popc(b[t]);
        }
        __syncthreads();
    }
}

__global__ void add_total_kernel(unsigned long long *m, const uint64_t *total)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *m += *total;
}

}  // namespace

Status launch_draw_movement(uint64_t n, uint64_t seed, double phi_lo, double phi_hi, double r_lo, double r_hi,
                            double *tau_phi, double *tau_r, cudaStream_t stream)
{
    Status st;
    if (!n) return st;
    draw_movement_kernel<<<grid(n), kThreads, 0, stream>>>(n, seed, phi_lo, phi_hi - phi_lo, r_lo, r_hi - r_lo,
                                                           tau_phi, tau_r);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_move(const uint32_t *ids, uint64_t count, uint64_t n, double *phi, double *r, const double *tau_phi,
                   double *tau_r, double R, double alpha, cudaStream_t stream)
{
    Status st;
    if (!count) return st;
    move_kernel<<<grid(count), kThreads, 0, stream>>>(ids, count, n, phi, r, tau_phi, tau_r, R, alpha);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_mark_moved(const uint32_t *ids, uint64_t count, uint64_t n, uint8_t *moved_by_id,
                         uint32_t *moved_bits, cudaStream_t stream)
{
    Status st;
    fill_u8_kernel<<<grid(n), kThreads, 0, stream>>>(moved_by_id, n, 0);
    RHG_LAUNCH_CHECK();
    fill_u32_kernel<<<grid(ceil_div(n, 32)), kThreads, 0, stream>>>(moved_bits, ceil_div(n, 32));
    RHG_LAUNCH_CHECK();
    if (count) {
        mark_kernel<<<grid(count), kThreads, 0, stream>>>(ids, count, n, moved_by_id, moved_bits);
        RHG_LAUNCH_CHECK();
    }
    return st;
}

Status launch_owners(const Meta *M, const uint32_t *sorted_ids, uint64_t n, const uint8_t *moved_by_id,
                     uint8_t *moved_by_pos, uint32_t *owners, uint64_t cap, unsigned long long *counter,
                     cudaStream_t stream)
{
    Status st;
    owners_kernel<<<grid(n), kThreads, 0, stream>>>(M, sorted_ids, n, moved_by_id, moved_by_pos, owners, cap, counter);
    RHG_LAUNCH_CHECK();
    return st;
}

size_t scan_temp_bytes(uint64_t count) { return (ceil_div(count ? count : 1, kScanBlock) + 1) * sizeof(uint64_t); }

Status launch_scan(const uint32_t *in, uint64_t count, uint64_t *out, void *temp, cudaStream_t stream)
{
    Status st;
    const uint64_t blocks = ceil_div(count ? count : 1, kScanBlock);
    uint64_t *sums = static_cast<uint64_t *>(temp);
    scan_sums_kernel<<<static_cast<unsigned>(blocks), kThreads, 0, stream>>>(in, count, sums);
    RHG_LAUNCH_CHECK();
    scan_top_kernel<<<1, kThreads, 0, stream>>>(sums, blocks);
    RHG_LAUNCH_CHECK();
    scan_apply_kernel<<<static_cast<unsigned>(blocks), kThreads, 0, stream>>>(in, count, sums, out);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_keep_old(const uint32_t *old_pairs, uint64_t m_old, const uint32_t *moved_bits, uint64_t n,
                       uint32_t *out, uint64_t cap, unsigned long long *counter, cudaStream_t stream)
{
    Status st;
    if (!m_old) return st;
    keep_old_kernel<<<grid(ceil_div(m_old, kKeepItems), 8), kThreads, 0, stream>>>(
        reinterpret_cast<const uint2 *>(old_pairs), m_old, moved_bits, n, reinterpret_cast<uint2 *>(out), cap,
        counter);
    RHG_LAUNCH_CHECK();
    return st;
}

Status launch_add_total(unsigned long long *m, const uint64_t *total, cudaStream_t stream)
{
    Status st;
    add_total_kernel<<<1, 32, 0, stream>>>(m, total);
    RHG_LAUNCH_CHECK();
    return st;
}

}  // namespace rhg
