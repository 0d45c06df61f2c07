// kernels.h -- host-side launchers of the CUDA path, one group per translation
// unit.  Each launcher enqueues its kernels on `stream` and returns a Status.
#pragma once
#include "common.cuh"

namespace rhg {

struct PlanArgs {
    uint64_t n;
    double k, alpha;
    uint64_t seed;
    uint32_t B;
    double p;
    double R_override;
    uint32_t allow_filter;  // FP32 filter permitted (the plan still requires R, alpha R in range)
    uint32_t verify;        // check every filter decision against the FP64 predicate
    uint32_t batch_budget, core_heavy, fringe_limit;  // work mapping of the range query (resolved, nonzero)
    uint32_t *bucket_counts;  // bucket_entries(n) counters the plan clears (bucket sort), or NULL
};

// Sorted, structure-of-arrays view of the points: position p is the p-th point in
// (band, angle key) order.  Filter mode fills akey/ang/pms/id; FP64 mode fills
// akey/id and phi/r/ch/sh.
struct SortedPoints {
    uint64_t n;
    const uint64_t *key;  // (band << 32) | angle key, ascending
    uint32_t *akey;       // angle key (low 32 bits of key)
    uint32_t *id;         // vertex id
    float2 *ang;          // filter: angle as hi + lo floats
    float4 *pms;          // filter: P, M, S, relative error of S
    double *phi;          // FP64 angle
    double *r;            // FP64 radius
    double *ch;           // dm::cosh(r)
    double *sh;           // dm::sinh(r)
};

// A batch of independent graphs (rhg_generate_batch): graph g owns the global
// positions [pt_off[g], pt_off[g+1]) of every per-point array, the bucket-index
// entries [idx_base[g], idx_base[g+1]) and the output pairs [out_off[g],
// out_off[g+1]).  Work is cut into tiles of at most kTilePoints positions that
// never cross a graph: tiles[t] = {graph, first position, count, 0}, and graph g's
// tiles are [tile_first[g], tile_first[g+1]).  Meta blocks: metas[g] per graph and
// metas[G], the control block holding the batch-wide counters and lists.
constexpr uint32_t kTilePoints = 2048;
struct BatchTables {
    uint32_t G;
    uint32_t num_tiles;
    const uint4 *tiles;
    const uint32_t *tile_first;  // G + 1
    const uint32_t *pt_off;      // G + 1
    const uint32_t *idx_base;    // G + 1
    const uint64_t *out_off;     // G + 1
    const uint32_t *bk_base;     // G + 1: the first sort bucket of each graph (bucket_entries(n) each)
};

// Everything the range query kernels read and write.
struct QueryArgs {
    Meta *M;                // the graph's Meta; batch: the G + 1 Meta blocks
    BatchTables bt;         // batch only
    SortedPoints P;
    const double *src_phi;  // caller points by id (rhg_edges_from_points), else NULL
    const double *src_r;
    uint32_t *pairs;        // output: pairs (u < v), or
    uint64_t *csr_keys;     // output: directed (row << 32 | col) keys, two per edge
    uint64_t capacity;      // output capacity in edges
    uint4 *heavy;           // heavy-range chunks {owner position, lo, hi, 0}
    uint32_t heavy_cap;
    uint2 *recheck;         // uncertain pairs {owner position, candidate position}
    uint32_t recheck_cap;
    uint32_t heavy_min;     // ranges longer than this go to the heavy chunks (UINT32_MAX: never)
    uint32_t *bidx;         // bucket index of the bands, index_entries(n) entries
    bool verify;            // some graph runs in verification mode (RHG_FLAG_VERIFY)
    uint32_t batch_lo, batch_hi;  // single graph: the warp batches [batch_lo, batch_hi) (batch_hi 0: all)
};

// ---- points.cu ----
Status launch_plan(Meta *d_meta, const PlanArgs &a, cudaStream_t stream);
// bucket_counts (optional): the sort buckets' point counts (bucket sort).
Status launch_sample(Meta *d_meta, uint64_t n, uint64_t seed, uint64_t *keys, uint32_t *ids,
                     double *r_by_id, uint32_t *bucket_counts, cudaStream_t stream);
Status launch_load_points(Meta *d_meta, uint64_t n, const double *phi, const double *r,
                          uint64_t *keys, uint32_t *ids, cudaStream_t stream);
Status launch_band_offsets(Meta *d_meta, cudaStream_t stream);
// Both gathers are launched; the one Meta::filter does not select returns at once.
// Filter: FP32 arrays (phi_src/r_src: caller points, else Philox).  FP64 mode:
// phi/r/ch/sh (r64_src: the sampled FP64 radii by id, or the caller radii).
Status launch_gather(const Meta *d_meta, uint64_t n, uint64_t seed, const uint64_t *sorted_keys,
                     const uint32_t *sorted_ids, const double *phi_src, const double *r_src,
                     const double *r64_src, SortedPoints P, cudaStream_t stream);
Status launch_dm_eval(int fn, const double *in, double *out, uint64_t count, cudaStream_t stream);
Status launch_points_by_id(const Meta *d_meta, uint64_t n, uint64_t seed, double *phi, double *r,
                           cudaStream_t stream);


// ---- bucket.cu ----
// Bucket sort of the keys (band << 32 | angle key) of points 0..n-1 by (key, id)
// (Alg. 1, angular sort within each band), for generated points, whose angles are
// uniform within a band: counts per bucket (the sampler's, or
// launch_bucket_count), an exclusive scan into bucket starts (with the band
// offsets of band_offsets_one), a scatter of (angle key << 32 | id) into the
// buckets, then one CTA per bucket sorts it in shared memory (a counting pass on
// the next 8 key bits, then each sub-bucket by one thread; buckets beyond
// kBucketCap or with a sub-bucket beyond kSubMax take an LSD radix sort of the
// bucket in global memory) and hands every position on: gather mode writes the
// sorted key back into comp and the filter (or FP64) values of the point
// (SortedPoints), keys mode writes the sorted keys and ids.
struct BucketArgs {
    Meta *M;
    uint64_t n;
    uint64_t seed;
    uint32_t *counts;        // bucket_entries(n): counts, then cursors
    uint32_t *start;         // bucket_entries(n) + 1: bucket starts
    uint64_t *comp;          // n: (angle key << 32 | id) by bucket; gather mode: the sorted keys after
    uint64_t *scratch;       // n: scratch of the global-memory path
    const double *r_by_id;   // FP64 mode: the sampled FP64 radii by id
    SortedPoints P;          // gather mode output
    uint64_t *out_keys;      // keys mode output
    uint32_t *out_ids;
};
Status launch_bucket_count(const BucketArgs &a, const uint64_t *keys, cudaStream_t stream);
// band offsets + bucket starts (one CTA)
Status launch_bucket_scan(const BucketArgs &a, cudaStream_t stream);
Status launch_bucket_scatter(const BucketArgs &a, const uint64_t *keys, cudaStream_t stream);
Status launch_bucket_sort(const BucketArgs &a, bool gather, cudaStream_t stream);

// ---- sort.cu ----
// LSD radix sort of 64-bit keys (optionally with uint32 values) over the 8-bit
// digits whose shifts are listed.  Stable.  On return *keys_out / *vals_out point at
// whichever buffer holds the result.  Temporary storage: radix_temp_bytes(n).
size_t radix_temp_bytes(uint64_t n);
Status radix_sort(uint64_t n, uint64_t *keys, uint64_t *keys_alt, uint32_t *vals,
                  uint32_t *vals_alt, const int *shifts, int num_shifts, void *temp,
                  uint64_t **keys_out, uint32_t **vals_out, cudaStream_t stream);


// ---- query.cu ----
// Range query (Alg. 1): windows, search, candidate test, output; then the heavy
// chunks and the FP64 rechecks.  Output positions are reserved per warp batch,
// so the pair order is unspecified; Meta::m is the exact edge count.  The kernels
// of both modes are launched; each returns at once unless Meta::filter selects it.
Status launch_query(const QueryArgs &a, bool csr, cudaStream_t stream);
// The range query in phases (pairs output): the bucket index, then for each phase
// a range of warp batches (the outermost sixteenth first, then the rest in equal
// parts inwards), their heavy chunks and FP64 rechecks; after phase p the edges
// [0, m) are final, m goes to
// Meta::m_phase[p] and, when host_m is not NULL (device pointer of mapped host
// memory), to host_m[p] as well.  events[p] (if not NULL) is recorded after phase p.
Status launch_query_phased(QueryArgs a, uint32_t phases, uint64_t *host_m, cudaEvent_t *events,
                           cudaStream_t stream);
// The whole batch in one persistent, cooperative launch: plan, sampling, band
// offsets, the segmented radix sort, gather, bucket index, both query phases and
// the per-graph results, separated by grid barriers whose waits give up after
// timeout_ns (the control block's error becomes kErrTimeout).  bar: 256 bytes of
// device memory, cleared here before the launch.  The caller's stage events
// cannot bracket stages inside one kernel; the control block records the device
// time of each stage instead (Meta::stage_ns, kBatchStageMarks entries).
struct PersistBuffers {
    Meta *metas;                 // G + 1 blocks (control block last)
    const PlanArgs *args;        // G
    BatchTables bt;
    uint64_t *keys0;             // sort keys by position (sampling), then the bucket sort's scratch
    uint64_t *keys1;             // composites by bucket, then the sorted keys (P.key)
    double *r_by_pos;            // FP64 radius by position (FP64 mode)
    uint32_t *bk_counts;         // bucket counts, then the scatter's cursors (bk_base[G] entries)
    uint32_t *bk_start;          // bucket starts (bk_base[G] + 1 entries)
    uint32_t *bk_info;           // bucket -> graph << 6 | band, or ~0 for an unused slot (bk_base[G] entries)
    SortedPoints P;              // gather output (P.key = keys1)
    uint32_t *pairs;
    uint4 *heavy;
    uint32_t heavy_cap;
    uint2 *recheck;
    uint32_t recheck_cap;
    uint32_t *bidx;
    uint4 *results;              // 2 G
    uint32_t *bar;               // grid barrier words
    uint64_t timeout_ns;
};
// stage marks a persistent launch records: start, plan, sampling, band offsets +
// bucket starts, bucket scatter, bucket sort + gather, bucket index, filter-mode
// query, its heavy chunks, rechecks, phase reset, FP64-mode query, its heavy
// chunks, results (the last mark is CTA 0's end)
constexpr int kBatchStages = 14;
Status launch_batch_persistent(const PersistBuffers &b, bool verify, cudaStream_t stream);
// One grid barrier on its own, for the test of the timeout: `missing` CTAs more
// than the launch has are expected, so with missing > 0 every wait runs out.
Status launch_barrier_test(Meta *C, uint32_t *bar, uint32_t missing, uint64_t timeout_ns, cudaStream_t stream);

// Bucket index alone (the subset query needs it without the full query).
Status launch_bucket_index(const QueryArgs &a, cudaStream_t stream);
// Neighbours of the moved vertices (dynamic model): counts (emit = false) or
// pairs at *base + offsets[slot] (emit = true); counts / offsets hold count * B
// (vertex, band) slots, then chunk_cap chunk slots; see subset_kernel.
Status launch_subset_query(const QueryArgs &a, const uint32_t *owners, uint64_t count,
                           const unsigned long long *owners_found, uint4 *chunks, uint64_t chunk_cap,
                           unsigned long long *chunk_n, const uint8_t *moved_by_pos, uint32_t *counts,
                           const uint64_t *offsets, const unsigned long long *base, uint64_t capacity, bool emit,
                           cudaStream_t stream);
// CSR row pointers from directed keys sorted by (row, col); col = low words.
Status launch_csr_finish(const uint64_t *sorted_keys, uint64_t entries, uint64_t n, uint64_t *row_ptr,
                         uint32_t *col, cudaStream_t stream);

// ---- dynamic.cu ----
Status launch_draw_movement(uint64_t n, uint64_t seed, double phi_lo, double phi_hi, double r_lo, double r_hi,
                            double *tau_phi, double *tau_r, cudaStream_t stream);
Status launch_move(const uint32_t *ids, uint64_t count, uint64_t n, double *phi, double *r, const double *tau_phi,
                   double *tau_r, double R, double alpha, cudaStream_t stream);
Status launch_mark_moved(const uint32_t *ids, uint64_t count, uint64_t n, uint8_t *moved_by_id,
                         uint32_t *moved_bits, cudaStream_t stream);
Status launch_owners(const Meta *M, const uint32_t *sorted_ids, uint64_t n, const uint8_t *moved_by_id,
                     uint8_t *moved_by_pos, uint32_t *owners, uint64_t cap, unsigned long long *counter,
                     cudaStream_t stream);
size_t scan_temp_bytes(uint64_t count);
// out[0..count) = exclusive prefix sums of in, out[count] = the total
Status launch_scan(const uint32_t *in, uint64_t count, uint64_t *out, void *temp, cudaStream_t stream);
Status launch_keep_old(const uint32_t *old_pairs, uint64_t m_old, const uint32_t *moved_bits, uint64_t n,
                       uint32_t *out, uint64_t cap, unsigned long long *counter, cudaStream_t stream);
Status launch_add_total(unsigned long long *m, const uint64_t *total, cudaStream_t stream);

}  // namespace rhg
