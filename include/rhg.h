/*
 * rhg.h -- C ABI of the GB300 generator of threshold random hyperbolic graphs
 * (band-based neighbour query of von Looz, Ozdayi, Laue, Meyerhenke,
 * "Generating massive complex networks with hyperbolic geometry faster in
 * practice", arXiv:1606.09481).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named d_* are device pointers on the CUDA device that is current
 *   for the calling thread; pointers named h_* (and every struct pointer) are
 *   host pointers.  The library never frees or retains caller memory.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Device work is enqueued on it in order; an entry point that
 *   returns a count to the host (m, R) synchronises that stream once, after the
 *   count is known.
 * - The caller provides all device memory: a workspace whose size
 *   rhg_workspace_bytes() (or the entry point's own sizing call) reports, and
 *   the output buffers.  Inside an entry point the library allocates no device
 *   memory; rhg_generate_batch and rhg_batch_prepare stage their per-graph
 *   tables in temporary host memory, the other entry points allocate none.
 * - Vertex ids are the Philox counter indices 0..n-1 (uint32).  An edge {u,v}
 *   is reported once as the pair (u, v) with u < v; the order of pairs is
 *   unspecified.  CSR rows list both directions with ascending columns.
 * - Every entry point returns an rhg_status.  Invalid arguments are reported
 *   before any device work; nothing aborts the process.  After RHG_ERR_CUDA the
 *   CUDA context may be unusable (the failing CUDA error is in
 *   rhg_result.cuda_error when a result pointer was given).
 *
 * The model (all FP64):
 * - alpha > 1/2, k > 0, 2 <= n <= 2^32 - 1.  R solves Krioukov's Eq. 22 for
 *   average degree k (paper Sec. III-B, getTargetRadius), unless R_override > 0.
 * - Point i: phi_i ~ U[0, 2pi), r_i by inverse CDF of Eq. 1 (Sec. II and
 *   Alg. 1), both from Philox4x64-10 with counter (i,0,0,0) and key (seed,0).
 * - Bands: num_bands rings with geometric boundaries of ratio band_ratio
 *   (Sec. III-A; defaults ceil(log2 n) and 0.9).
 * - Edge {v,w} iff the FP64 value cosh r_v cosh r_w - sinh r_v sinh r_w
 *   cos|phi_v - phi_w| is <= cosh R (Eq. 3 and the threshold test of Alg. 1),
 *   evaluated as one fixed sequence of rounded IEEE operations with the
 *   library's deterministic exp/log/cos; the edge set is therefore a pure
 *   function of (n, k, alpha, seed) and does not depend on num_bands,
 *   band_ratio or the filter flags.
 * - By default (R <= 32 and alpha R <= 44) an FP32 test decides each candidate
 *   pair whenever its proven error bound, which includes the rounding of the FP64
 *   predicate, allows; the remaining pairs are decided by the FP64 predicate.
 */
#ifndef RHG_H
#define RHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rhg_status {
    RHG_OK = 0,
    RHG_ERR_INVALID_ARG = 1,  /* a parameter or buffer is outside its domain          */
    RHG_ERR_NO_SOLUTION = 2,  /* no R gives average degree k (Eq. 22 peaks below k)   */
    RHG_ERR_OOM = 3,          /* the workspace passed is smaller than required, or a
                                 work list of the workspace overflowed (a graph far
                                 denser than its sizing assumed, e.g. num_bands = 1
                                 on a large n)                                        */
    RHG_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed          */
    RHG_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up                   */
    RHG_ERR_OVERFLOW = 6      /* the output buffer holds fewer entries than required;
                                 rhg_result.m reports the exact edge count            */
} rhg_status;

#define RHG_MAX_BANDS 64u

/* flags */
#define RHG_FLAG_FP64_ONLY 0x1u  /* evaluate every candidate with the FP64 predicate
                                    (no FP32 filter); same edge set, slower          */
#define RHG_FLAG_VERIFY 0x2u     /* debugging: also evaluate the FP64 predicate for
                                    every pair the FP32 filter decides, and count
                                    disagreements in rhg_result.verify_failures
                                    (must be 0); much slower                         */

/* Parameters of one graph (Alg. 1 input: n, average degree k, alpha = (gamma-1)/2). */
typedef struct rhg_params {
    uint64_t n;          /* vertices, 2 <= n <= 2^32 - 1                              */
    double k;            /* target average degree (Eq. 22), > 0                       */
    double alpha;        /* radial dispersion, > 1/2 and <= 100; gamma = 2 alpha + 1  */
    uint64_t seed;       /* Philox key word 0                                         */
    uint32_t num_bands;  /* 0 = ceil(log2 n); otherwise 1..64 (Sec. III-A)            */
    uint32_t flags;      /* RHG_FLAG_*                                                */
    double band_ratio;   /* 0 = 0.9; otherwise > 0 (Sec. III-A, ratio p)              */
    double R_override;   /* > 0: use this disk radius instead of solving Eq. 22       */
    /* Work mapping of the range query (performance only, never the edge set);
     * 0 = the library default:                                                   */
    uint32_t batch_budget; /* candidates one warp batch of 32 points keeps before
                              its longer ranges go to the shared chunk list
                              (default 65536; 1024 .. 2^24)                        */
    uint32_t core_heavy;   /* longest certain range a warp batch writes itself
                              (default 4096; 64 .. 65536)                          */
    uint32_t fringe_limit; /* longest tested range a lane tests itself
                              (default 32; 1 .. 32)                                */
    uint32_t reserved;     /* must be 0                                           */
} rhg_params;

/* Per-call report, filled on the host when the pointer is non-NULL. */
typedef struct rhg_result {
    uint64_t m;               /* undirected edges of the graph (exact, also on OVERFLOW) */
    double R;                 /* disk radius used                                        */
    uint32_t num_bands;       /* bands used                                              */
    int32_t cuda_error;       /* cudaError_t of the failing call when status is CUDA     */
    uint64_t candidates;      /* candidate pairs examined by the range query             */
    uint64_t near_threshold;  /* candidates with |L - cosh R| <= 1e-12 cosh R            */
    uint64_t rechecks;        /* candidates the FP32 filter sent to the FP64 predicate   */
    uint64_t verify_failures; /* RHG_FLAG_VERIFY: filter decisions the FP64 predicate
                                 contradicts (0 unless the filter's error bound fails) */
    uint32_t mode;            /* 1: FP32 filter + FP64 recheck; 0: FP64 predicate only */
    uint32_t heavy_chunks;    /* long candidate ranges split across warps (diagnostic)  */
    uint64_t rounding_band;   /* candidates with |L - cosh R| <= 8 u cosh r_v cosh r_w
                                 (u = 2^-53): the pairs whose decision the rounding of
                                 Eq. 3 in FP64 can flip (diagnostic)                   */
} rhg_result;

/* Human-readable name of a status code (static string, never NULL). */
const char *rhg_status_str(int status);

/* ABI version of this header: 4 (2 added rhg_result.rounding_band, 3 the work
 * mapping fields of rhg_params, 4 rhg_sort_keys and the batch's bucket-sort
 * stages in rhg_batch_stage_times). */
int rhg_version(void);

/*
 * rhg_default_bands -- the band count used when rhg_params.num_bands is 0:
 * ceil(log2 n), at least 1 (the "log n" bands of Sec. III-A).  Host-only; n = 0
 * and 1 give 1.
 */
uint32_t rhg_default_bands(uint64_t n);

/*
 * rhg_plan_workspace_bytes -- device workspace rhg_target_radius and rhg_plan
 * need (a few KB of per-graph metadata).  Host-only.
 */
size_t rhg_plan_workspace_bytes(void);

/*
 * rhg_target_radius -- R such that Eq. 22 (Krioukov et al., with zeta = 1) gives
 * average degree k (paper Sec. III-B, getTargetRadius): the largest integer
 * grid point j in [0, 255] with kbar(j) > k brackets the crossing, then binary
 * search until the bracket holds adjacent doubles; R is the upper end, the
 * smallest double found with kbar(R) <= k.  Runs one kernel on `stream` in
 * d_workspace (>= rhg_plan_workspace_bytes()) and synchronises the stream.
 * Errors: INVALID_ARG (n, k, alpha out of domain, NULL pointer), OOM (workspace
 * too small), NO_SOLUTION, CUDA.
 */
int rhg_target_radius(uint64_t n, double k, double alpha, void *d_workspace, size_t workspace_bytes,
                      void *stream, double *R_out);

/*
 * rhg_plan -- R and the band boundaries c_0 = 0 < c_1 < ... < c_B = R that
 * rhg_generate_* use for these parameters (Sec. III-A; c_{j+1} - c_j =
 * c_1 p^j, c_1 = (1-p) R / (1-p^B)).  Computed on the device in d_workspace
 * (>= rhg_plan_workspace_bytes()); synchronises the stream.  h_c receives
 * B + 1 doubles (it must hold RHG_MAX_BANDS + 1); *num_bands_out receives B.
 */
int rhg_plan(const rhg_params *p, void *d_workspace, size_t workspace_bytes, void *stream, double *R_out,
             double *h_c, uint32_t *num_bands_out);

/*
 * rhg_workspace_bytes -- device workspace that rhg_generate_pairs needs for p
 * (capacity_entries = 0) or that rhg_generate_csr needs for an output of
 * capacity_entries directed column entries.  Host-only; no device work.
 */
int rhg_workspace_bytes(const rhg_params *p, uint64_t capacity_entries, size_t *bytes);

/*
 * rhg_sample_points -- the points of Alg. 1 (its sampling step), by id:
 * d_phi[i], d_r[i] for i < n (FP64; Philox4x64-10, inverse CDF of Eq. 1).
 * d_workspace must hold rhg_plan_workspace_bytes().  Writes R to *R_out and
 * synchronises the stream.
 */
int rhg_sample_points(const rhg_params *p, void *d_workspace, size_t workspace_bytes,
                      double *d_phi, double *d_r, void *stream, double *R_out);

/*
 * rhg_generate_pairs -- the whole hot path of Alg. 1 on the device: R, band
 * boundaries, sampling, band assignment, radix sort by (band, phi), windows
 * (getMinMaxPhi), binary search, candidate test, and compaction of the edges
 * into d_pairs as m pairs (u, v), u < v, uint32 (2 m words, 8-byte aligned;
 * d_workspace 256-byte aligned).  capacity_edges is the number of pairs d_pairs
 * holds; if m exceeds it, d_pairs holds an unspecified subset and the call
 * returns RHG_ERR_OVERFLOW with result->m = m (call again with room for m).
 */
int rhg_generate_pairs(const rhg_params *p, void *d_workspace, size_t workspace_bytes,
                       uint32_t *d_pairs, uint64_t capacity_edges, void *stream,
                       rhg_result *result);

/*
 * rhg_generate_pairs_host -- rhg_generate_pairs followed by a copy of the m
 * pairs into host memory h_pairs (2 * h_capacity_edges uint32 words; pinned
 * memory makes the copy asynchronous-capable).  Synchronises the stream.
 * OVERFLOW if m exceeds either capacity.
 */
int rhg_generate_pairs_host(const rhg_params *p, void *d_workspace, size_t workspace_bytes,
                            uint32_t *d_pairs, uint64_t capacity_edges, uint32_t *h_pairs,
                            uint64_t h_capacity_edges, void *stream, rhg_result *result);

/*
 * rhg_generate_pairs_static -- rhg_generate_pairs without a caller workspace and
 * without allocating device memory.  The paper has no counterpart: this is a
 * library convenience.  It serves callers that cannot allocate device memory,
 * such as code that runs under a device-memory budget fixed up front, a plugin
 * whose host program owns every device allocation, or a loop that cannot afford
 * the device-wide synchronisation a cudaFree implies.
 *
 * The scratch is one fixed array of RHG_STATIC_SCRATCH_BYTES in the library's
 * device image, so p->n is limited to RHG_STATIC_MAX_POINTS; a larger n, or a
 * graph whose workspace (rhg_workspace_bytes) exceeds the scratch (a dense graph
 * that may run in FP64 mode, whose chunk list grows with n k), returns
 * RHG_ERR_INVALID_ARG before anything is launched.  The array's address is
 * looked up by the first call in each CUDA context (the current device's primary
 * context, or the caller's own; a context created again after cudaDeviceReset
 * gets a new lookup), so that first call should come before any stream capture
 * begins.  Like rhg_generate_pairs, every call ends with a synchronisation of
 * `stream` to read back the edge count.  Nothing in the
 * scratch has to start at zero: the first kernel of every call resets the
 * counters it uses.  All calls on one device share the one array, so calls
 * that overlap in time (other host threads, or other streams before the
 * previous call returned) race; serialise them.  d_pairs, capacity_edges,
 * result and the return codes are as in rhg_generate_pairs, and the edges are
 * the same.
 */
#define RHG_STATIC_MAX_POINTS 131072u
#define RHG_STATIC_SCRATCH_BYTES (16u << 20)
int rhg_generate_pairs_static(const rhg_params *p, uint32_t *d_pairs, uint64_t capacity_edges,
                              void *stream, rhg_result *result);

/*
 * rhg_generate_csr -- the same graph as symmetric CSR: d_row_ptr (n + 1 uint64)
 * and d_col (2 m uint32, ascending within each row).  capacity_entries is the
 * number of uint32 d_col holds; the workspace must hold
 * rhg_workspace_bytes(p, capacity_entries).  OVERFLOW if 2 m > capacity_entries.
 */
int rhg_generate_csr(const rhg_params *p, void *d_workspace, size_t workspace_bytes,
                     uint64_t *d_row_ptr, uint32_t *d_col, uint64_t capacity_entries,
                     void *stream, rhg_result *result);

/*
 * rhg_edges_from_points -- the range query of Alg. 1 on caller-given points
 * (d_phi[i] in [0, 2pi), d_r[i] in [0, R], FP64, by id) with disk radius R:
 * bands, sort, windows, candidate test and compaction, as in
 * rhg_generate_pairs.  The workspace must hold rhg_workspace_bytes_points(n,
 * num_bands).  Points outside the domain give INVALID_ARG.
 */
int rhg_workspace_bytes_points(uint64_t n, uint32_t num_bands, size_t *bytes);
int rhg_edges_from_points(const double *d_phi, const double *d_r, uint64_t n, double R,
                          uint32_t num_bands, double band_ratio, uint32_t flags,
                          void *d_workspace, size_t workspace_bytes, uint32_t *d_pairs,
                          uint64_t capacity_edges, void *stream, rhg_result *result);

/*
 * Batches of independent graphs (the batched workload: thousands of small graphs
 * of uneven size generated together).  Each graph is exactly the graph that
 * rhg_generate_pairs gives for the same rhg_params (same R, points, bands and
 * edge set); only the work is shared: one launch of each stage covers every
 * graph (sampling, a sort segmented by graph, gather, range query).
 *
 * rhg_batch_workspace_bytes -- workspace bytes rhg_generate_batch needs for
 * these `count` graphs (it depends on the n of each graph, not on the output).
 *
 * rhg_generate_batch -- graphs[g] (n >= 2, k, alpha, seed, num_bands, band_ratio,
 * R_override, flags as in rhg_params) for g < count.  Graph g writes its pairs
 * (u < v, vertex ids 0 .. n_g - 1 of that graph, order unspecified) to
 * d_pairs[2 pair_offsets[g] ..], with room for pair_offsets[g + 1] -
 * pair_offsets[g] pairs; pair_offsets is a host array of count + 1
 * non-decreasing entries and d_pairs holds pair_offsets[count] pairs (8-byte
 * aligned).  results (host, count entries) receives each graph's exact edge
 * count, R, band count, mode (1 = FP32 filter + FP64 recheck) and status:
 * RHG_ERR_OVERFLOW when its edges exceed its room (call again with room for
 * results[g].m), RHG_ERR_NO_SOLUTION when its k cannot be reached, else RHG_OK.
 * totals (optional) receives the sum of the edges of the graphs with status
 * RHG_OK and the batch-wide counters.  Returns RHG_OK when every graph
 * succeeded, else the status of the first graph that did not; argument errors
 * (including one invalid graph) return RHG_ERR_INVALID_ARG before any launch.
 * Limits: count <= 2^20 graphs and fewer than 2^32 points in all.  The tables
 * of the batch are copied from pageable host memory, and the call synchronises
 * the stream once at the end (twice when a list overflowed in filter mode and
 * the batch reran in FP64 mode).
 */
typedef struct {
    uint64_t m;           /* edges of the graph (exact, also on overflow)        */
    double R;             /* disk radius                                          */
    uint32_t num_bands;
    int32_t status;       /* RHG_OK, RHG_ERR_OVERFLOW, RHG_ERR_NO_SOLUTION, ...   */
    uint32_t mode;        /* 1: FP32 filter + FP64 recheck; 0: FP64 predicate     */
    uint32_t reserved;
} rhg_batch_graph;

int rhg_batch_workspace_bytes(const rhg_params *graphs, uint32_t count, size_t *bytes);
int rhg_generate_batch(const rhg_params *graphs, uint32_t count, void *d_workspace,
                       size_t workspace_bytes, uint32_t *d_pairs, const uint64_t *pair_offsets,
                       void *stream, rhg_batch_graph *results, rhg_result *totals);

/*
 * The same batch split into a host step and a capturable device step, so that
 * the device work can be recorded once in a CUDA graph and replayed.
 *
 * rhg_batch_prepare -- the host part of rhg_generate_batch (same arguments and
 * argument errors): checks the graphs, cuts them into tiles and copies the
 * per-graph tables into d_workspace (returns when the copy is done), and fills
 * *plan (host).  The tables stay valid in d_workspace until it is reused.
 *
 * rhg_batch_launch -- enqueues every stage of the prepared batch on `stream`:
 * kernel launches only, with no host memory, synchronisation or allocation, so
 * it may run inside stream capture (cudaStreamBeginCapture).  Each launch or
 * replay regenerates the same graphs into d_pairs (the layout of
 * rhg_generate_batch, pair_capacity = pair_offsets[count] pairs) and the
 * per-graph results into d_workspace.  plan must be the one rhg_batch_prepare
 * filled for this d_workspace; a plan whose counts do not describe a workspace
 * of plan->workspace_bytes returns RHG_ERR_INVALID_ARG.  Unlike
 * rhg_generate_batch it never reruns a batch in FP64 mode: if the FP64 recheck
 * list overflows, every graph reports RHG_ERR_OOM and rhg_generate_batch (which
 * reruns) is the fallback.
 *
 * rhg_batch_read_results -- waits for `stream`, then fills results (count
 * entries) and totals (optional) from the last launch, as rhg_generate_batch
 * does, and returns the same status.
 */
typedef struct {
    uint32_t count;            /* graphs                                        */
    uint32_t verify;           /* 1 if some graph has RHG_FLAG_VERIFY            */
    uint64_t num_tiles;        /* work tiles (at most 2048 points, one graph)   */
    uint64_t points;           /* points of all graphs                          */
    uint64_t index_entries;    /* bucket-index entries of all graphs            */
    uint64_t pair_capacity;    /* pair_offsets[count]                           */
    uint64_t workspace_bytes;  /* = rhg_batch_workspace_bytes of the graphs     */
    uint64_t chunk_extra;      /* chunk-list entries for graphs in FP64 mode    */
} rhg_batch_plan;

int rhg_batch_prepare(const rhg_params *graphs, uint32_t count, const uint64_t *pair_offsets,
                      void *d_workspace, size_t workspace_bytes, void *stream, rhg_batch_plan *plan);
int rhg_batch_launch(const rhg_batch_plan *plan, void *d_workspace, uint32_t *d_pairs, void *stream);
int rhg_batch_read_results(const rhg_batch_plan *plan, const void *d_workspace, void *stream,
                           rhg_batch_graph *results, rhg_result *totals);

/*
 * The batch runs as one persistent, cooperative kernel launch: all its stages,
 * one after another, each spread over every resident CTA, separated by grid
 * barriers.  A barrier wait gives up after 20 s of device time; the batch then
 * reports RHG_ERR_TIMEOUT (for every graph) instead of hanging the device.
 *
 * rhg_batch_stage_times -- device time of each stage of the last launch in
 * d_workspace (after the launch has completed), in ms, RHG_BATCH_STAGE_COUNT
 * values in this order: plan, sampling (with the sort-bucket counts), band
 * offsets and bucket starts, bucket scatter, bucket sort with the gather, bucket
 * index, range query (filter graphs), heavy chunks (filter graphs), FP64
 * rechecks, phase reset, range query (FP64 graphs), heavy chunks (FP64 graphs),
 * results.  Synchronises the stream.  Errors: INVALID_ARG (no plan, count too
 * small), CUDA.
 */
#define RHG_BATCH_STAGE_COUNT 13u
int rhg_batch_stage_times(const rhg_batch_plan *plan, const void *d_workspace, void *stream, double *ms,
                          uint32_t count);

/*
 * rhg_grid_barrier_test -- the grid barrier of the persistent batch launch on
 * its own, for testing its timeout: a cooperative launch of 2 CTAs per SM whose
 * barrier expects `missing` more CTAs than there are.  missing = 0: the barrier
 * completes, RHG_OK.  missing > 0: no CTA can pass, every wait gives up after
 * timeout_ns (at most 10 s) and the call returns RHG_ERR_TIMEOUT; the device
 * stays usable.  d_workspace: rhg_plan_workspace_bytes() + 256 bytes, 256-byte
 * aligned.  Synchronises the stream.
 */
int rhg_grid_barrier_test(uint32_t missing, uint64_t timeout_ns, void *d_workspace, size_t workspace_bytes,
                          void *stream);

/*
 * Dynamic model (Sec. III-C): vertices move in discrete steps, each a rotation
 * phi + tau_phi (mod 2 pi) and the radial movement of Algorithm 2 with
 * reflection, taken in the coordinate x = cosh(alpha r) - 1 (computed as
 * 2 sinh^2(alpha r / 2)): y = x + tau_r, mirrored at cosh(alpha R) - 1 or at 0
 * while outside (tau_r changes sign: the vertex bounces), then
 * r = 2 asinh(sqrt(y / 2)) / alpha (at most R).  Theorem 1 (the positions keep
 * the density of Eq. 1) holds for a coordinate that is uniform under Eq. 1;
 * x is (its CDF is x / (cosh(alpha R) - 1)), while the sinh(alpha r) printed in
 * Algorithm 2 is not, and a walk in it drifts towards the centre.  All FP64, in
 * the fixed operation order of the library's deterministic functions.
 *
 * rhg_draw_movement -- step values of vertices 0 .. n-1 from Philox counter
 * (i, 1, 0, 0), key (seed, 0): tau_phi uniform in [phi_lo, phi_hi), tau_r
 * uniform in [r_lo, r_hi) (the paper's experiment: (-1, 1) and (-10, 1)).
 *
 * rhg_move_points -- one step of the `count` distinct vertices d_ids (ids < n)
 * on the FP64 coordinates d_phi, d_r (by id, in place; the result of
 * rhg_sample_points or of earlier steps), with step values d_tau_phi, d_tau_r
 * (tau_r's sign flips are written back).  INVALID_ARG for count > n or an
 * unusable R or alpha; ids at or above n are skipped.
 *
 * rhg_update_edges -- the edge list after a step, without generating the graph
 * again: d_old_pairs (m_old pairs u < v, the graph of these points before the
 * step, e.g. from rhg_edges_from_points or an earlier update) keeps the pairs
 * whose endpoints both stayed; the moved vertices d_moved_ids (the ids given to
 * rhg_move_points) are queried against all bands of the moved point set
 * (d_phi, d_r after the step, disk radius R), and their pairs are added, each
 * once.  The result in d_new_pairs (room for capacity_edges pairs, must not
 * overlap d_old_pairs) is, as a set, the graph rhg_edges_from_points gives for
 * the moved points.  Workspace: rhg_workspace_bytes_update(n, moved_count,
 * num_bands) (num_bands 0: the default, as in rhg_update_edges).
 * result->m = exact edge count (OVERFLOW when above the capacity); INVALID_ARG
 * when an id repeats or is out of range (detected on the device).
 */
int rhg_draw_movement(uint64_t n, uint64_t seed, double phi_lo, double phi_hi, double r_lo, double r_hi,
                      double *d_tau_phi, double *d_tau_r, void *stream);
int rhg_move_points(const uint32_t *d_ids, uint64_t count, uint64_t n, double *d_phi, double *d_r,
                    const double *d_tau_phi, double *d_tau_r, double R, double alpha, void *stream);
int rhg_workspace_bytes_update(uint64_t n, uint64_t moved_count, uint32_t num_bands, size_t *bytes);
int rhg_update_edges(const double *d_phi, const double *d_r, uint64_t n, double R, uint32_t num_bands,
                     double band_ratio, uint32_t flags, const uint32_t *d_moved_ids, uint64_t moved_count,
                     const uint32_t *d_old_pairs, uint64_t m_old, void *d_workspace, size_t workspace_bytes,
                     uint32_t *d_new_pairs, uint64_t capacity_edges, void *stream, rhg_result *result);

/*
 * rhg_sort_keys -- the angular sort of Alg. 1 (points by band, then by angle key
 * within the band) as the generator runs it on its own points, on caller keys:
 * d_keys[i] = (band << 32) | angle key of point i, band < num_bands; band j is
 * cut into 2^bucket_bits[j] buckets (bucket_bits[j] <= 24, a host array) by the
 * top bits of the angle key.  Writes d_sorted_keys (n uint64) and d_sorted_ids (n
 * uint32: the i of each key), ascending by (key, i).  Every key distribution is
 * sorted; a bucket of more than 2048 keys, or more than 32 keys of one bucket
 * sharing the next 8 angle-key bits, takes a slower path (the generator sizes its
 * buckets from the band's expected count: 512 to 1024 uniform angles each).
 * Workspace: rhg_sort_keys_workspace_bytes, 256-byte aligned.  Errors:
 * INVALID_ARG (arguments; a band >= num_bands in d_keys, found on the device),
 * OOM (workspace too small), CUDA.  Synchronises the stream.
 */
int rhg_sort_keys_workspace_bytes(uint64_t n, uint32_t num_bands, const uint32_t *bucket_bits, size_t *bytes);
int rhg_sort_keys(const uint64_t *d_keys, uint64_t n, uint32_t num_bands, const uint32_t *bucket_bits,
                  void *d_workspace, size_t workspace_bytes, uint64_t *d_sorted_keys, uint32_t *d_sorted_ids,
                  void *stream);

/*
 * rhg_dm_eval -- the library's deterministic FP64 functions on a device array,
 * for verification against an independent implementation: fn = 0 exp, 1 log,
 * 2 cos, 3 cosh, 4 sinh, 5 asinh (y >= 0; dynamic model).  d_out[i] = f(d_in[i]),
 * i < count.
 */
int rhg_dm_eval(int fn, const double *d_in, double *d_out, uint64_t count, void *stream);

/*
 * Profiling aids (not part of the method).
 *
 * rhg_set_stage_events -- when `events` is non-NULL, every later generate /
 * edges_from_points call records events[2 s] and events[2 s + 1] (cudaEvent_t
 * handles created by the caller, passed as void*) on its stream immediately
 * before and after stage s, for s < count / 2 and s < RHG_NUM_STAGES, so that
 * cudaEventElapsedTime gives each stage's device time.  Process-wide and not
 * thread-safe; NULL switches it off.  Stages that do not run record nothing.
 * Independently of this, every stage is an NVTX range ("rhg.plan",
 * "rhg.sample", "rhg.sort", "rhg.gather", "rhg.query", "rhg.csr") on the calling
 * thread, for Nsight tools.
 *
 * rhg_launch_count -- number of kernels this library has launched in this
 * process so far (all devices, all threads).
 */
#define RHG_STAGE_PLAN 0u     /* R solve and band boundaries                      */
#define RHG_STAGE_SAMPLE 1u   /* Philox sampling / point load and band histogram  */
#define RHG_STAGE_SORT 2u     /* band offsets and radix sort by (band, angle)     */
#define RHG_STAGE_GATHER 3u   /* sorted structure-of-arrays                       */
#define RHG_STAGE_QUERY 4u    /* range query: windows, search, test, emit, recheck */
#define RHG_STAGE_CSR 5u      /* CSR sort and row pointers                        */
#define RHG_NUM_STAGES 6u
int rhg_set_stage_events(void *const *events, uint32_t count);
uint64_t rhg_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* RHG_H */
