// kernels.h -- host-side launchers of the CUDA path, one group per translation
// unit.  Each launcher enqueues its kernels on `stream` and returns a Status.
#pragma once
#include "common.cuh"

namespace rhg {

// Sorted, structure-of-arrays view of the points: position p is the p-th point in
// (band, angle) order.
struct SortedPoints {
    uint64_t n;
    const uint64_t *key;  // (band << 32) | angle key, ascending
    double *phi;          // FP64 angle
    double *r;            // FP64 radius
    double *ch;           // dm::cosh(r)
    double *sh;           // dm::sinh(r)
    uint32_t *akey;       // angle key (low 32 bits of key)
    uint32_t *id;         // vertex id
};

// ---- points.cu ----
// Plan: R (Eq. 22 solve, or R_override > 0), boundaries, constants; zeroes counters.
Status launch_plan(Meta *d_meta, uint64_t n, double k, double alpha, uint64_t seed, uint32_t B,
                   double p, double R_override, cudaStream_t stream);
// Sample: Philox points by id, band of each, sort keys; band histogram.
Status launch_sample(Meta *d_meta, uint64_t n, uint64_t seed, uint64_t *keys, uint32_t *ids,
                     double *r_by_id, cudaStream_t stream);
// Load caller points (validates 0 <= phi < 2pi, 0 <= r <= R).
Status launch_load_points(Meta *d_meta, uint64_t n, const double *phi, const double *r,
                          uint64_t *keys, uint32_t *ids, cudaStream_t stream);
// Band offsets from the histogram.
Status launch_band_offsets(Meta *d_meta, cudaStream_t stream);
// Gather the sorted SoA (phi recomputed from Philox when phi_by_id is NULL).
Status launch_gather(const Meta *d_meta, uint64_t n, uint64_t seed, const uint64_t *sorted_keys,
                     const uint32_t *sorted_ids, const double *phi_by_id, const double *r_by_id,
                     SortedPoints P, cudaStream_t stream);
// rhg_dm_eval
Status launch_dm_eval(int fn, const double *in, double *out, uint64_t count, cudaStream_t stream);
// Sampled points by id (phi, r), for rhg_sample_points.
Status launch_points_by_id(const Meta *d_meta, uint64_t n, uint64_t seed, double *phi, double *r,
                           cudaStream_t stream);

// ---- sort.cu ----
// LSD radix sort of 64-bit keys (optionally with uint32 values) over the 8-bit
// digits whose shifts are listed.  Stable.  On return *keys_out / *vals_out point at
// whichever buffer holds the result.  Temporary storage: radix_temp_bytes(n).
size_t radix_temp_bytes(uint64_t n);
Status radix_sort(uint64_t n, uint64_t *keys, uint64_t *keys_alt, uint32_t *vals,
                  uint32_t *vals_alt, const int *shifts, int num_shifts, void *temp,
                  uint64_t **keys_out, uint32_t **vals_out, cudaStream_t stream);

// ---- query.cu ----
size_t scan_temp_bytes(uint64_t n);
// Exclusive scan of counts into offsets[0..n]; the total goes to *total_dst.
Status exclusive_scan_u32(const uint32_t *counts, uint64_t *offsets, uint64_t n, uint64_t *total_dst,
                          void *temp, cudaStream_t stream);
// Range query, count pass (per sorted position: edges reported from it).
Status launch_query_count(Meta *d_meta, SortedPoints P, uint32_t *counts, cudaStream_t stream);
// Range query, emit pass: pairs (u < v) at offsets, or directed CSR keys when csr != 0.
Status launch_query_emit(Meta *d_meta, SortedPoints P, const uint64_t *offsets, uint32_t *pairs,
                         uint64_t *csr_keys, cudaStream_t stream);
// CSR row pointers from directed keys sorted by (row, col); col = low words.
Status launch_csr_finish(const uint64_t *sorted_keys, uint64_t entries, uint64_t n, uint64_t *row_ptr,
                         uint32_t *col, cudaStream_t stream);

}  // namespace rhg
