// api.cu -- the extern "C" entry points declared in include/rhg.h: argument
// validation, workspace layout, and the stream-ordered pipeline
//   plan -> sample -> band offsets -> radix sort -> gather -> bucket index ->
//   range query (edges reserved per warp and band) -> FP64 recheck
//   [-> CSR sort/finish] -> one D2H of the metadata (m, R, counters).
#include <atomic>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

// A CUDA call in an entry point that reports through rhg_result: on failure the
// error goes to res->cuda_error and the entry returns RHG_ERR_CUDA.
#define RHG_RESULT_TRY(expr, res)          \
    do {                                   \
        const cudaError_t _e = (expr);     \
        if (_e != cudaSuccess) {           \
            (res)->cuda_error = _e;        \
            return RHG_ERR_CUDA;           \
        }                                  \
    } while (0)

namespace rhg {

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

// rhg_set_stage_events state (profiling aid, process-wide)
void *const *g_events = nullptr;
uint32_t g_num_events = 0;

// Stage boundaries: an NVTX range per stage on the calling thread (seen by
// Nsight tools; a few nanoseconds without one) and, when rhg_set_stage_events
// is on, the caller's events on the stream.
void mark(uint32_t stage, bool end, cudaStream_t s)
{
    static const char *const kStageNames[RHG_NUM_STAGES] = {"rhg.plan", "rhg.sample", "rhg.sort",
                                                            "rhg.gather", "rhg.query", "rhg.csr"};
    thread_local nvtxRangeId_t open[RHG_NUM_STAGES] = {};
    if (stage < RHG_NUM_STAGES) {
        if (!end) {
            open[stage] = nvtxRangeStartA(kStageNames[stage]);
        } else if (open[stage]) {
            nvtxRangeEnd(open[stage]);
            open[stage] = 0;
        }
    }
    const uint32_t i = 2 * stage + (end ? 1 : 0);
    if (g_events && i < g_num_events && g_events[i])
        cudaEventRecord(static_cast<cudaEvent_t>(g_events[i]), s);
}

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Byte offsets of every buffer inside the caller's workspace.
struct Layout {
    size_t meta, keys0, keys1, ids0, ids1, r_by_id, akey, id, ang, pms, phi, r, ch, sh, heavy, recheck, bidx,
        bcount, bstart, sort_tmp, csr0, csr1, total;
    uint32_t heavy_cap, recheck_cap;
};

constexpr uint64_t kMaxListEntries = 0x7fffffffull;

// Work mapping of the range query: rhg_params' fields, 0 meaning these defaults.
constexpr uint32_t kDefaultBatchBudget = 65536, kDefaultCoreHeavy = 4096, kDefaultFringeLimit = 32;

// Eq. 22 (zeta = 1) in plain double arithmetic, for host-side sizing only (the
// device plan computes the R the graph uses).
double host_kbar(double R, double n, double a)
{
    const double pi = 3.14159265358979323846, xi = a / (a - 0.5);
    const double inner = pi / (4.0 * a * a) - (pi - 1.0) / a + (pi - 2.0);
    return 2.0 / pi * xi * xi * n * (std::exp(-R / 2.0) + std::exp(-a * R) * (a * R / 2.0 * inner - 1.0));
}

// R of Eq. 22 for sizing: the decreasing-branch solution by bisection, as the
// device plan does it (largest integer j in [0, 255] with kbar(j) > k, then
// bisection); within ~1e-12 of the device's R.  0 when there is no solution.
double host_radius_estimate(const rhg_params &p)
{
    if (p.R_override > 0.0) return p.R_override;
    const double n = static_cast<double>(p.n);
    // the e^{-R/2} term alone gives R to within a few units; far from the filter's
    // limits that decides the sizing without the bisection (a batch sizes
    // thousands of graphs on the host)
    const double pi = 3.14159265358979323846, xi = p.alpha / (p.alpha - 0.5);
    const double lead = 2.0 * std::log(2.0 / pi * xi * xi * n / p.k);
    if (lead < kFilterMaxR - 6.0 && p.alpha * lead < kFilterMaxAlphaR - 6.0 * p.alpha) return lead;
    int j = -1;
    for (int t = 0; t < 256; ++t)
        if (host_kbar(t, n, p.alpha) > p.k) j = t;
    if (j < 0 || j == 255) return 0.0;
    double lo = j, hi = j + 1.0;
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (host_kbar(mid, n, p.alpha) > p.k) lo = mid;
        else hi = mid;
    }
    return hi;
}

// Chunk-list entries beyond n/4 + 65536 for a graph that may run in FP64 mode
// (RHG_FLAG_FP64_ONLY, or R > 32 or alpha R > 44, which decide the mode on the
// device; R solved from Eq. 22 on the host, with a margin of 0.25 for the
// difference to the device's R): without a core every window is tested, and
// each tested piece longer than 32 candidates becomes at least one chunk, so the
// list is sized by the candidates, about 1.1-2 times the n k / 2 edges:
// n k / 20 entries, with k from Eq. 22 at R for an R_override.
uint64_t fp64_chunk_extra(const rhg_params &p)
{
    const double R = host_radius_estimate(p);
    const bool fp64 = (p.flags & RHG_FLAG_FP64_ONLY) != 0 || R > kFilterMaxR - 0.25 ||
                      p.alpha * R > kFilterMaxAlphaR - 0.25;
    const double k = p.R_override > 0.0 ? host_kbar(p.R_override, static_cast<double>(p.n), p.alpha) : p.k;
    if (!fp64 || !(k > 0.0)) return 0;
    const double extra = std::ceil(static_cast<double>(p.n) * k / 20.0);
    return extra < static_cast<double>(kMaxListEntries) ? static_cast<uint64_t>(extra) : kMaxListEntries;
}

// Chunk-list entries beyond the defaults' sizing for a graph whose work mapping
// sends more pieces to the chunk list: every piece pushed holds more candidates
// than its limit, and the candidates are at most about 1.2 times the n k / 2
// edges, so each smaller limit L adds 0.6 n k / (L + 1) entries.
uint64_t mapping_chunk_extra(const rhg_params &p)
{
    double k = p.k;
    if (p.R_override > 0.0) k = host_kbar(p.R_override, static_cast<double>(p.n), p.alpha);
    if (!(k > 0.0)) return 0;
    const double nk = 0.6 * static_cast<double>(p.n) * k;
    double extra = 0.0;
    if (p.fringe_limit && p.fringe_limit < kDefaultFringeLimit) extra += nk / (p.fringe_limit + 1.0);
    uint32_t core = p.core_heavy ? p.core_heavy : kDefaultCoreHeavy;
    if (p.batch_budget && p.batch_budget / 32 < core) core = p.batch_budget / 32 > 64 ? p.batch_budget / 32 : 64;
    if (core < kDefaultCoreHeavy) extra += nk / (core + 1.0);
    extra = std::ceil(extra);
    return extra < static_cast<double>(kMaxListEntries) ? static_cast<uint64_t>(extra) : kMaxListEntries;
}

uint64_t chunk_extra(const rhg_params &p)
{
    const uint64_t e = fp64_chunk_extra(p) + mapping_chunk_extra(p);
    return e < kMaxListEntries ? e : kMaxListEntries;
}

Layout make_layout(uint64_t n, uint64_t csr_entries, uint64_t chunk_extra = 0)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const uint64_t chunks = n / 4 + 65536 + chunk_extra;
    L.heavy_cap = static_cast<uint32_t>(chunks < kMaxListEntries ? chunks : kMaxListEntries);
    L.recheck_cap = static_cast<uint32_t>(n / 2 + 65536);
    L.meta = take(sizeof(Meta));
    L.keys0 = take(n * 8);
    L.keys1 = take(n * 8);
    L.ids0 = take(n * 4);
    L.ids1 = take(n * 4);
    L.r_by_id = take(n * 8);
    L.akey = take(n * 4);
    L.id = take(n * 4);
    L.ang = take(n * 8);
    L.pms = take(n * 16);
    L.phi = take(n * 8);
    L.r = take(n * 8);
    L.ch = take(n * 8);
    L.sh = take(n * 8);
    L.heavy = take(static_cast<size_t>(L.heavy_cap) * 16);
    L.recheck = take(static_cast<size_t>(L.recheck_cap) * 8);
    L.bidx = take(static_cast<size_t>(index_entries(n)) * 4);
    L.bcount = take(static_cast<size_t>(bucket_entries(n)) * 4);
    L.bstart = take(static_cast<size_t>(bucket_entries(n) + 1) * 4);
    const size_t sort_points = radix_temp_bytes(n);
    const size_t sort_csr = csr_entries ? radix_temp_bytes(csr_entries) : 0;
    L.sort_tmp = take(sort_points > sort_csr ? sort_points : sort_csr);
    L.csr0 = take(csr_entries * 8);
    L.csr1 = take(csr_entries * 8);
    L.total = o;
    return L;
}

template <typename T>
T *at(void *base, size_t off)
{
    return reinterpret_cast<T *>(static_cast<char *>(base) + off);
}

uint32_t default_bands(uint64_t n)
{
    uint32_t B = 0;
    while (B < 63 && (uint64_t{1} << B) < n) ++B;
    return B < 1 ? 1 : B;
}

constexpr uint32_t kKnownFlags = RHG_FLAG_FP64_ONLY | RHG_FLAG_VERIFY;


PlanArgs with_mapping(PlanArgs pa, uint32_t budget, uint32_t core_heavy, uint32_t fringe)
{
    pa.batch_budget = budget ? budget : kDefaultBatchBudget;
    pa.core_heavy = core_heavy ? core_heavy : kDefaultCoreHeavy;
    pa.fringe_limit = fringe ? fringe : kDefaultFringeLimit;
    return pa;
}

PlanArgs with_mapping(PlanArgs pa, const rhg_params &p)
{
    return with_mapping(pa, p.batch_budget, p.core_heavy, p.fringe_limit);
}

// Host-side validation of rhg_params; fills B and p.
int check_params(const rhg_params *p, uint32_t *B, double *ratio)
{
    if (!p) return RHG_ERR_INVALID_ARG;
    if (p->n < 2 || p->n > 0xFFFFFFFFull) return RHG_ERR_INVALID_ARG;
    if (!(p->alpha > 0.5) || !(p->alpha <= 100.0)) return RHG_ERR_INVALID_ARG;
    const bool has_R = p->R_override > 0.0;
    if (has_R && !(std::isfinite(p->R_override) && p->R_override <= 700.0)) return RHG_ERR_INVALID_ARG;
    if (!has_R && !(p->k > 0.0 && p->k < 1e300)) return RHG_ERR_INVALID_ARG;
    if (p->num_bands > RHG_MAX_BANDS) return RHG_ERR_INVALID_ARG;
    if (p->band_ratio < 0.0 || !std::isfinite(p->band_ratio)) return RHG_ERR_INVALID_ARG;
    if (p->flags & ~kKnownFlags) return RHG_ERR_INVALID_ARG;
    if (p->reserved) return RHG_ERR_INVALID_ARG;
    if (p->batch_budget && (p->batch_budget < 1024 || p->batch_budget > (1u << 24))) return RHG_ERR_INVALID_ARG;
    if (p->core_heavy && (p->core_heavy < 64 || p->core_heavy > 65536)) return RHG_ERR_INVALID_ARG;
    if (p->fringe_limit > 32) return RHG_ERR_INVALID_ARG;
    *B = p->num_bands ? p->num_bands : default_bands(p->n);
    *ratio = p->band_ratio > 0.0 ? p->band_ratio : 0.9;
    return RHG_OK;
}

int finish(const Status &st, rhg_result *res)
{
    if (res && st.code == RHG_ERR_CUDA) res->cuda_error = static_cast<int32_t>(st.cuda);
    return st.code;
}

int error_from_meta(uint32_t e)
{
    switch (e) {
        case kErrNone: return RHG_OK;
        case kErrNoSolution: return RHG_ERR_NO_SOLUTION;
        case kErrBadPoint: return RHG_ERR_INVALID_ARG;
        case kErrTimeout: return RHG_ERR_TIMEOUT;
        case kErrListFull: return RHG_ERR_OOM;
        default: return RHG_ERR_CUDA;
    }
}

Status read_meta(const Meta *d_meta, Meta *h, cudaStream_t stream)
{
    Status st;
    RHG_CUDA_TRY(cudaMemcpyAsync(h, d_meta, sizeof(Meta), cudaMemcpyDeviceToHost, stream));
    RHG_CUDA_TRY(cudaStreamSynchronize(stream));
    return st;
}

void fill_result(rhg_result *res, const Meta &h)
{
    if (!res) return;
    res->m = h.m;
    res->R = h.R;
    res->num_bands = h.B;
    res->candidates = h.candidates;
    res->near_threshold = h.near_threshold;
    res->rounding_band = h.rounding_band;
    res->rechecks = h.rechecks;
    res->verify_failures = h.verify_failures;
    res->mode = h.filter ? 1u : 0u;
    res->heavy_chunks = h.heavy_n;
}

struct Pipeline {
    void *ws;
    Layout L;
    uint64_t n;
    Meta *meta() const { return at<Meta>(ws, L.meta); }
    SortedPoints sorted(const uint64_t *sorted_keys) const
    {
        SortedPoints P;
        P.n = n;
        P.key = sorted_keys;
        P.akey = at<uint32_t>(ws, L.akey);
        P.id = at<uint32_t>(ws, L.id);
        P.ang = at<float2>(ws, L.ang);
        P.pms = at<float4>(ws, L.pms);
        P.phi = at<double>(ws, L.phi);
        P.r = at<double>(ws, L.r);
        P.ch = at<double>(ws, L.ch);
        P.sh = at<double>(ws, L.sh);
        return P;
    }
};

int bits_for(uint64_t v)
{
    int b = 0;
    while (b < 64 && (v >> b)) ++b;
    return b;
}

enum class Output { Pairs, Csr };

// The point pipeline on the stream: plan, points, bands, sort, gather.
Status enqueue_points(const Pipeline &pl, const PlanArgs &pa, const double *phi_in, const double *r_in,
                      SortedPoints *P_out, cudaStream_t stream)
{
    Status st;
    Meta *M = pl.meta();
    uint64_t *k0 = at<uint64_t>(pl.ws, pl.L.keys0), *k1 = at<uint64_t>(pl.ws, pl.L.keys1);
    uint32_t *i0 = at<uint32_t>(pl.ws, pl.L.ids0), *i1 = at<uint32_t>(pl.ws, pl.L.ids1);
    double *rid = at<double>(pl.ws, pl.L.r_by_id);
    if (!phi_in) {
        // generated points (uniform angles): bucket sort with the gather fused in
        BucketArgs ba{};
        ba.M = M;
        ba.n = pl.n;
        ba.seed = pa.seed;
        ba.counts = at<uint32_t>(pl.ws, pl.L.bcount);
        ba.start = at<uint32_t>(pl.ws, pl.L.bstart);
        ba.comp = k1;
        ba.scratch = k0;
        ba.r_by_id = rid;
        ba.P = pl.sorted(k1);
        PlanArgs pb = pa;
        pb.bucket_counts = ba.counts;
        mark(RHG_STAGE_PLAN, false, stream);
        st = launch_plan(M, pb, stream);
        if (st.code) return st;
        mark(RHG_STAGE_PLAN, true, stream);
        mark(RHG_STAGE_SAMPLE, false, stream);
        st = launch_sample(M, pl.n, pa.seed, k0, nullptr, rid, ba.counts, stream);
        if (st.code) return st;
        mark(RHG_STAGE_SAMPLE, true, stream);
        mark(RHG_STAGE_SORT, false, stream);
        st = launch_bucket_scan(ba, stream);
        if (st.code) return st;
        st = launch_bucket_scatter(ba, k0, stream);
        if (st.code) return st;
        mark(RHG_STAGE_SORT, true, stream);
        mark(RHG_STAGE_GATHER, false, stream);
        st = launch_bucket_sort(ba, true, stream);
        if (st.code) return st;
        mark(RHG_STAGE_GATHER, true, stream);
        *P_out = ba.P;
        return st;
    }
    mark(RHG_STAGE_PLAN, false, stream);
    st = launch_plan(M, pa, stream);
    if (st.code) return st;
    mark(RHG_STAGE_PLAN, true, stream);
    mark(RHG_STAGE_SAMPLE, false, stream);
    st = launch_load_points(M, pl.n, phi_in, r_in, k0, i0, stream);
    if (st.code) return st;
    mark(RHG_STAGE_SAMPLE, true, stream);
    mark(RHG_STAGE_SORT, false, stream);
    st = launch_band_offsets(M, stream);
    if (st.code) return st;
    // key = (band << 32) | angle key; band < 64 needs 6 more bits
    const int shifts[5] = {0, 8, 16, 24, 32};
    uint64_t *ks = nullptr;
    uint32_t *is = nullptr;
    st = radix_sort(pl.n, k0, k1, i0, i1, shifts, 5, at<void>(pl.ws, pl.L.sort_tmp), &ks, &is, stream);
    if (st.code) return st;
    mark(RHG_STAGE_SORT, true, stream);
    mark(RHG_STAGE_GATHER, false, stream);
    const SortedPoints P = pl.sorted(ks);
    st = launch_gather(M, pl.n, pa.seed, ks, is, phi_in, r_in, phi_in ? r_in : rid, P, stream);
    if (st.code) return st;
    mark(RHG_STAGE_GATHER, true, stream);
    *P_out = P;
    return st;
}

// One full pass of the hot path on the stream: the point pipeline, then the range
// query (+ heavy chunks + FP64 rechecks).  No host synchronisation.
Status enqueue(const Pipeline &pl, const PlanArgs &pa, const double *phi_in, const double *r_in, Output kind,
               uint32_t *d_pairs, uint64_t capacity_edges, uint32_t heavy_min, cudaStream_t stream)
{
    SortedPoints P;
    Status st = enqueue_points(pl, pa, phi_in, r_in, &P, stream);
    if (st.code) return st;
    Meta *M = pl.meta();
    QueryArgs q{};
    q.M = M;
    q.P = P;
    q.src_phi = phi_in;
    q.src_r = r_in;
    q.pairs = kind == Output::Pairs ? d_pairs : nullptr;
    q.csr_keys = kind == Output::Csr ? at<uint64_t>(pl.ws, pl.L.csr0) : nullptr;
    q.capacity = capacity_edges;
    q.heavy = at<uint4>(pl.ws, pl.L.heavy);
    q.heavy_cap = pl.L.heavy_cap;
    q.recheck = at<uint2>(pl.ws, pl.L.recheck);
    q.recheck_cap = pl.L.recheck_cap;
    q.heavy_min = heavy_min;
    q.bidx = at<uint32_t>(pl.ws, pl.L.bidx);
    q.verify = pa.verify != 0;
    mark(RHG_STAGE_QUERY, false, stream);
    st = launch_query(q, kind == Output::Csr, stream);
    if (st.code) return st;
    mark(RHG_STAGE_QUERY, true, stream);
    return st;
}

constexpr uint32_t kHeavyMin = 256;

// Runs the pipeline and reads the metadata back (one synchronisation).  If the
// FP64-recheck list overflowed it runs again in FP64 mode, which needs none; a
// heavy-chunk list that overflows even then (average degree in the thousands)
// is reported as RHG_ERR_OOM by the caller.
Status run_pipeline(const Pipeline &pl, PlanArgs pa, const double *phi_in, const double *r_in, Output kind,
                    uint32_t *d_pairs, uint64_t capacity_edges, Meta *h, cudaStream_t stream)
{
    Status st = enqueue(pl, pa, phi_in, r_in, kind, d_pairs, capacity_edges, kHeavyMin, stream);
    if (st.code) return st;
    st = read_meta(pl.meta(), h, stream);
    if (st.code) return st;
    if (h->error == kErrListFull && h->filter) {
        pa.allow_filter = 0;
        st = enqueue(pl, pa, phi_in, r_in, kind, d_pairs, capacity_edges, kHeavyMin, stream);
        if (st.code) return st;
        st = read_meta(pl.meta(), h, stream);
    }
    return st;
}

int generate(const rhg_params *p, void *d_ws, size_t ws_bytes, Output kind, uint32_t *d_pairs, uint64_t capacity,
             uint64_t *d_row_ptr, uint32_t *d_col, cudaStream_t stream, rhg_result *res)
{
    if (res) std::memset(res, 0, sizeof(*res));
    uint32_t B;
    double ratio;
    int rc = check_params(p, &B, &ratio);
    if (rc) return rc;
    if (!d_ws) return RHG_ERR_INVALID_ARG;
    if (kind == Output::Pairs && capacity && (!d_pairs || (reinterpret_cast<uintptr_t>(d_pairs) & 7)))
        return RHG_ERR_INVALID_ARG;
    if (kind == Output::Csr && (!d_row_ptr || (capacity && !d_col))) return RHG_ERR_INVALID_ARG;
    const Layout L = make_layout(p->n, kind == Output::Csr ? capacity : 0, chunk_extra(*p));
    if (ws_bytes < L.total) return RHG_ERR_OOM;
    if (reinterpret_cast<uintptr_t>(d_ws) & 255) return RHG_ERR_INVALID_ARG;
    Pipeline pl{d_ws, L, p->n};
    PlanArgs pa = with_mapping(PlanArgs{p->n, p->k, p->alpha, p->seed, B, ratio, p->R_override,
                                        (p->flags & RHG_FLAG_FP64_ONLY) ? 0u : 1u,
                                        (p->flags & RHG_FLAG_VERIFY) ? 1u : 0u},
                               *p);
    const uint64_t cap_edges = kind == Output::Pairs ? capacity : capacity / 2;
    Meta h;
    Status st = run_pipeline(pl, pa, nullptr, nullptr, kind, d_pairs, cap_edges, &h, stream);
    if (st.code) return finish(st, res);
    fill_result(res, h);
    if (h.error) return error_from_meta(h.error);
    if (h.m > cap_edges) return RHG_ERR_OVERFLOW;
    if (kind == Output::Csr) {
        const uint64_t entries = 2 * h.m;
        uint64_t *c0 = at<uint64_t>(pl.ws, pl.L.csr0), *c1 = at<uint64_t>(pl.ws, pl.L.csr1);
        const int nb = bits_for(p->n - 1);
        int shifts[16];
        int ns = 0;
        for (int s = 0; s < nb; s += 8) shifts[ns++] = s;
        for (int s = 0; s < nb; s += 8) shifts[ns++] = 32 + s;
        uint64_t *sorted = nullptr;
        mark(RHG_STAGE_CSR, false, stream);
        st = radix_sort(entries, c0, c1, nullptr, nullptr, shifts, ns, at<void>(pl.ws, pl.L.sort_tmp), &sorted,
                        nullptr, stream);
        if (st.code) return finish(st, res);
        st = launch_csr_finish(sorted, entries, p->n, d_row_ptr, d_col, stream);
        if (st.code) return finish(st, res);
        mark(RHG_STAGE_CSR, true, stream);
        const cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            st.code = RHG_ERR_CUDA;
            st.cuda = e;
            return finish(st, res);
        }
    }
    return RHG_OK;
}

// ------------------------------------------------------------------ batch
constexpr uint32_t kMaxBatch = 1u << 20;
// A grid barrier of the persistent batch launch that waits longer than this
// gives up: the batch then returns RHG_ERR_TIMEOUT instead of hanging the device.
constexpr uint64_t kBatchTimeoutNs = 20ull * 1000 * 1000 * 1000;

// Host-side tables of a batch (uploaded once per call).
struct BatchHost {
    uint32_t G = 0;
    uint64_t N = 0;          // points of all graphs
    uint64_t idx_total = 0;  // bucket-index entries of all graphs
    uint64_t chunk_extra = 0;  // chunk-list entries for graphs that may run in FP64 mode
    std::vector<PlanArgs> args;
    std::vector<uint4> tiles;
    std::vector<uint32_t> tile_first, pt_off, idx_base, bk_base;
    std::vector<uint64_t> out_off;
};

struct BatchLayout {
    size_t metas, args, tiles, tile_first, pt_off, idx_base, bk_base, out_off, tables_end, results, keys0, keys1,
        r_by_pos, akey, id, ang, pms, phi, r, ch, sh, bidx, bk_counts, bk_start, bk_info, heavy, recheck, bar, total;
    uint32_t heavy_cap, recheck_cap;
};

// Sort buckets of a batch: graph g owns n_g / kBucketTarget + B_g + 1 of them, so
// all graphs together own at most this many (from the point and graph counts alone).
uint64_t batch_buckets(uint64_t G, uint64_t N) { return N / kBucketTarget + G * (kMaxBands + 1); }

int batch_host(const rhg_params *graphs, uint32_t count, const uint64_t *pair_offsets, BatchHost &h)
{
    if (!graphs || count == 0 || count > kMaxBatch) return RHG_ERR_INVALID_ARG;
    h.G = count;
    h.args.resize(count);
    h.tile_first.assign(count + 1, 0);
    h.pt_off.assign(count + 1, 0);
    h.idx_base.assign(count + 1, 0);
    h.bk_base.assign(count + 1, 0);
    h.out_off.assign(count + 1, 0);
    h.tiles.clear();
    uint64_t pos = 0, idx = 0;
    for (uint32_t g = 0; g < count; ++g) {
        const rhg_params &q = graphs[g];
        uint32_t B;
        double ratio;
        const int rc = check_params(&q, &B, &ratio);
        if (rc) return rc;
        h.args[g] = with_mapping(PlanArgs{q.n, q.k, q.alpha, q.seed, B, ratio, q.R_override,
                                          (q.flags & RHG_FLAG_FP64_ONLY) ? 0u : 1u,
                                          (q.flags & RHG_FLAG_VERIFY) ? 1u : 0u},
                                 q);
        h.tile_first[g] = static_cast<uint32_t>(h.tiles.size());
        for (uint64_t s0 = 0; s0 < q.n; s0 += kTilePoints) {
            const uint64_t c = q.n - s0 < kTilePoints ? q.n - s0 : kTilePoints;
            h.tiles.push_back(make_uint4(g, static_cast<uint32_t>(pos + s0), static_cast<uint32_t>(c), 0u));
        }
        pos += q.n;
        idx += index_entries(q.n);
        h.chunk_extra += chunk_extra(q);
        if (pos >= 0xFFFFFFFFull || idx >= 0xFFFFFFFFull) return RHG_ERR_INVALID_ARG;  // 32-bit positions
        h.pt_off[g + 1] = static_cast<uint32_t>(pos);
        h.idx_base[g + 1] = static_cast<uint32_t>(idx);
        // the plan's buckets: 2^b per band with 2^b <= E / kBucketTarget, so at most
        // n / kBucketTarget + B of them, and one more start
        h.bk_base[g + 1] = static_cast<uint32_t>(h.bk_base[g] + q.n / kBucketTarget + B + 1);
    }
    h.tile_first[count] = static_cast<uint32_t>(h.tiles.size());
    h.N = pos;
    h.idx_total = idx;
    if (pair_offsets) {
        for (uint32_t g = 0; g <= count; ++g) {
            if (g && pair_offsets[g] < pair_offsets[g - 1]) return RHG_ERR_INVALID_ARG;
            h.out_off[g] = pair_offsets[g];
        }
    }
    return RHG_OK;
}

// Byte offsets of a batch's buffers from its graph, point, tile and index counts.
BatchLayout batch_layout(uint64_t G, uint64_t N, uint64_t num_tiles, uint64_t idx_total, uint64_t chunk_extra)
{
    BatchLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const uint64_t chunks = N / 4 + 65536 + chunk_extra;
    L.heavy_cap = static_cast<uint32_t>(chunks < kMaxListEntries ? chunks : kMaxListEntries);
    L.recheck_cap = static_cast<uint32_t>(N / 2 + 65536);
    L.metas = take((G + 1) * sizeof(Meta));
    // the tables are one contiguous upload
    L.args = o;
    o += G * sizeof(PlanArgs);
    o = (o + 15) & ~size_t{15};
    L.tiles = o;
    o += num_tiles * sizeof(uint4);
    L.tile_first = o;
    o += (G + 1) * 4;
    L.pt_off = o;
    o += (G + 1) * 4;
    L.idx_base = o;
    o += (G + 1) * 4;
    L.bk_base = o;
    o += (G + 1) * 4;
    o = (o + 7) & ~size_t{7};
    L.out_off = o;
    o += (G + 1) * 8;
    L.tables_end = o;
    o = align_up(o);
    L.results = take(2 * G * sizeof(uint4));
    L.keys0 = take(N * 8);
    L.keys1 = take(N * 8);
    L.r_by_pos = take(N * 8);
    L.akey = take(N * 4);
    L.id = take(N * 4);
    L.ang = take(N * 8);
    L.pms = take(N * 16);
    L.phi = take(N * 8);
    L.r = take(N * 8);
    L.ch = take(N * 8);
    L.sh = take(N * 8);
    L.bidx = take(idx_total * 4);
    L.bk_counts = take(batch_buckets(G, N) * 4);
    L.bk_start = take((batch_buckets(G, N) + 1) * 4);
    L.bk_info = take(batch_buckets(G, N) * 4);
    L.heavy = take(static_cast<size_t>(L.heavy_cap) * 16);
    L.recheck = take(static_cast<size_t>(L.recheck_cap) * 8);
    L.bar = take(256);
    L.total = o;
    return L;
}

BatchLayout batch_layout(const BatchHost &h)
{
    return batch_layout(h.G, h.N, h.tiles.size(), h.idx_total, h.chunk_extra);
}

// Copies the tables into the workspace (pageable source: returns when copied).
Status upload_tables(void *ws, const BatchLayout &L, const BatchHost &h, cudaStream_t stream)
{
    Status st;
    std::vector<unsigned char> buf(L.tables_end - L.args, 0);
    auto put = [&](size_t off, const void *src, size_t bytes) {
        if (bytes) std::memcpy(buf.data() + (off - L.args), src, bytes);
    };
    // each graph's plan clears its own bucket counters
    std::vector<PlanArgs> args = h.args;
    for (uint32_t g = 0; g < h.G; ++g) args[g].bucket_counts = at<uint32_t>(ws, L.bk_counts) + h.bk_base[g];
    put(L.args, args.data(), args.size() * sizeof(PlanArgs));
    put(L.tiles, h.tiles.data(), h.tiles.size() * sizeof(uint4));
    put(L.tile_first, h.tile_first.data(), h.tile_first.size() * 4);
    put(L.pt_off, h.pt_off.data(), h.pt_off.size() * 4);
    put(L.idx_base, h.idx_base.data(), h.idx_base.size() * 4);
    put(L.bk_base, h.bk_base.data(), h.bk_base.size() * 4);
    put(L.out_off, h.out_off.data(), h.out_off.size() * 8);
    RHG_CUDA_TRY(cudaMemcpyAsync(at<char>(ws, L.args), buf.data(), buf.size(), cudaMemcpyHostToDevice, stream));
    RHG_CUDA_TRY(cudaStreamSynchronize(stream));
    return st;
}

BatchTables batch_tables(void *ws, const BatchLayout &L, uint32_t G, uint64_t num_tiles)
{
    BatchTables bt;
    bt.G = G;
    bt.num_tiles = static_cast<uint32_t>(num_tiles);
    bt.tiles = at<uint4>(ws, L.tiles);
    bt.tile_first = at<uint32_t>(ws, L.tile_first);
    bt.pt_off = at<uint32_t>(ws, L.pt_off);
    bt.idx_base = at<uint32_t>(ws, L.idx_base);
    bt.out_off = at<uint64_t>(ws, L.out_off);
    bt.bk_base = at<uint32_t>(ws, L.bk_base);
    return bt;
}

// Every stage of the batch on the stream, in one persistent cooperative launch
// (plan of all graphs, sampling, band offsets, segmented sort, gather, bucket
// index, range query, results; launch_batch_persistent).  No host memory and no
// synchronisation, so the launch can be captured into a CUDA graph.
Status enqueue_batch(void *ws, const BatchLayout &L, uint32_t G, uint64_t N, uint64_t num_tiles, bool verify,
                     uint32_t *d_pairs, cudaStream_t stream)
{
    PersistBuffers b{};
    b.metas = at<Meta>(ws, L.metas);
    b.args = at<PlanArgs>(ws, L.args);
    b.bt = batch_tables(ws, L, G, num_tiles);
    b.keys0 = at<uint64_t>(ws, L.keys0);
    b.keys1 = at<uint64_t>(ws, L.keys1);
    b.r_by_pos = at<double>(ws, L.r_by_pos);
    b.bk_counts = at<uint32_t>(ws, L.bk_counts);
    b.bk_start = at<uint32_t>(ws, L.bk_start);
    b.bk_info = at<uint32_t>(ws, L.bk_info);
    SortedPoints &P = b.P;
    P.n = N;
    P.key = b.keys1;  // the bucket sort writes the sorted keys back over its composites
    P.akey = at<uint32_t>(ws, L.akey);
    P.id = at<uint32_t>(ws, L.id);
    P.ang = at<float2>(ws, L.ang);
    P.pms = at<float4>(ws, L.pms);
    P.phi = at<double>(ws, L.phi);
    P.r = at<double>(ws, L.r);
    P.ch = at<double>(ws, L.ch);
    P.sh = at<double>(ws, L.sh);
    b.pairs = d_pairs;
    b.heavy = at<uint4>(ws, L.heavy);
    b.heavy_cap = L.heavy_cap;
    b.recheck = at<uint2>(ws, L.recheck);
    b.recheck_cap = L.recheck_cap;
    b.bidx = at<uint32_t>(ws, L.bidx);
    b.results = at<uint4>(ws, L.results);
    b.bar = at<uint32_t>(ws, L.bar);
    b.timeout_ns = kBatchTimeoutNs;
    return launch_batch_persistent(b, verify, stream);
}

bool any_verify(const BatchHost &h)
{
    for (const PlanArgs &g : h.args)
        if (g.verify) return true;
    return false;
}

// Per-graph results and totals from the device results table (two uint4 per
// graph), the batch's control block and the pair offsets.
int fill_batch_results(uint32_t count, const uint4 *res, const Meta &ctl, const uint64_t *out_off,
                       rhg_batch_graph *results, rhg_result *totals)
{
    int rc = RHG_OK;
    uint64_t total_m = 0;
    uint32_t all_filter = 1;
    for (uint32_t g = 0; g < count; ++g) {
        const uint4 a = res[2 * g], b = res[2 * g + 1];
        rhg_batch_graph &r = results[g];
        r.m = static_cast<uint64_t>(a.x) | (static_cast<uint64_t>(a.y) << 32);
        const uint64_t Rb = static_cast<uint64_t>(a.z) | (static_cast<uint64_t>(a.w) << 32);
        std::memcpy(&r.R, &Rb, sizeof(double));
        r.num_bands = b.x;
        r.mode = b.z ? 1u : 0u;
        r.status = ctl.error ? error_from_meta(ctl.error) : error_from_meta(b.y);
        if (r.status == RHG_OK && r.m > out_off[g + 1] - out_off[g]) r.status = RHG_ERR_OVERFLOW;
        if (r.status == RHG_OK) total_m += r.m;
        if (!r.mode) all_filter = 0;
        if (rc == RHG_OK && r.status != RHG_OK) rc = r.status;
    }
    if (totals) {
        totals->m = total_m;
        totals->candidates = ctl.candidates;
        totals->near_threshold = ctl.near_threshold;
        totals->rounding_band = ctl.rounding_band;
        totals->rechecks = ctl.rechecks;
        totals->verify_failures = ctl.verify_failures;
        totals->heavy_chunks = ctl.heavy_n;
        totals->mode = all_filter;
    }
    return rc;
}

// ------------------------------------------------------------------ dynamic
// Workspace of rhg_update_edges: the point pipeline of the moved points, then
// the moved flags (by id and by sorted position), the moved vertices' sorted
// positions, their pair counts, offsets and the scan's block sums.
struct UpdateLayout {
    Layout L;
    size_t moved_id, moved_bits, moved_pos, owners, counts, offsets, scan_tmp, chunks, total;
    uint64_t chunk_cap;
};

UpdateLayout update_layout(uint64_t n, uint64_t moved, uint32_t B)
{
    UpdateLayout U{};
    U.L = make_layout(n, 0);
    size_t o = U.L.total;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    U.chunk_cap = 2 * moved + 65536;
    const uint64_t slots = moved * B + U.chunk_cap;
    U.moved_id = take(n);
    U.moved_bits = take(ceil_div(n, 32) * 4);
    U.moved_pos = take(n);
    U.owners = take(moved * 4);
    U.counts = take(slots * 4);
    U.offsets = take((slots + 1) * 8);
    U.scan_tmp = take(scan_temp_bytes(slots));
    U.chunks = take(U.chunk_cap * 16);
    U.total = o;
    return U;
}

// Scratch of rhg_generate_pairs_static: one array in the device image, found by
// symbol.  Each CUDA context (the primary context of each device, a new primary
// context after cudaDeviceReset, a caller's own context) loads its own copy of
// the image, so the address is looked up once per context and cached under the
// context's unique id (cuCtxGetId), reached through the runtime's driver entry
// points so that the library needs no link to the driver library.
__device__ __align__(256) unsigned char g_static_scratch[RHG_STATIC_SCRATCH_BYTES];
constexpr int kMaxContexts = 64;
std::mutex g_static_mu;
unsigned long long g_static_ctx[kMaxContexts] = {};  // context ids (0: unused slot)
void *g_static_ptr[kMaxContexts] = {};
int g_static_next = 0;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Id of the calling thread's current context (0 if there is none yet).
int current_context_id(unsigned long long *id, cudaError_t *err)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {  // under g_static_mu
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        *err = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (*err == cudaSuccess)
            *err = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (*err != cudaSuccess) return RHG_ERR_CUDA;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            *err = cudaErrorNotSupported;
            return RHG_ERR_CUDA;
        }
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    *id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS) {
        *err = cudaErrorDeviceUninitialized;
        return RHG_ERR_CUDA;
    }
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) {
        *err = cudaErrorDeviceUninitialized;
        return RHG_ERR_CUDA;
    }
    return RHG_OK;
}

// The current context's scratch address; the lookup runs once per context.
int static_scratch(void **ptr, cudaError_t *err)
{
    std::lock_guard<std::mutex> lock(g_static_mu);
    unsigned long long id = 0;
    int rc = current_context_id(&id, err);
    if (rc) return rc;
    for (int j = 0; id && j < kMaxContexts; ++j)
        if (g_static_ctx[j] == id) {
            *ptr = g_static_ptr[j];
            return RHG_OK;
        }
    void *a = nullptr;
    *err = cudaGetSymbolAddress(&a, g_static_scratch);  // makes the device's primary context current if none is
    if (*err != cudaSuccess) return RHG_ERR_CUDA;
    if (!id) {
        rc = current_context_id(&id, err);
        if (rc) return rc;
    }
    if (id) {  // slots are reused round robin once every slot has been taken
        g_static_ctx[g_static_next] = id;
        g_static_ptr[g_static_next] = a;
        g_static_next = (g_static_next + 1) % kMaxContexts;
    }
    *ptr = a;
    return RHG_OK;
}

// Resources of rhg_generate_pairs_host's overlapped copy, made once per CUDA
// context and kept: a copy stream, one event per query phase, and host words
// (registered, mapped) the phase ends write their edge counts into.  The mutex
// serialises the calls that use them.
struct HostCopy {
    std::mutex mu;
    cudaStream_t copy = nullptr;
    cudaEvent_t ev[kMaxPhases] = {};
    uint64_t *h_m = nullptr;  // this context's kMaxPhases words
    uint64_t *d_m = nullptr;  // their device address
};
alignas(4096) uint64_t g_phase_words[kMaxContexts][kMaxPhases];
bool g_phase_words_registered = false;
std::mutex g_copy_mu;
unsigned long long g_copy_ctx[kMaxContexts] = {};
HostCopy g_copy[kMaxContexts];

int host_copy_resources(HostCopy **out, cudaError_t *err)
{
    std::lock_guard<std::mutex> lock(g_copy_mu);
    unsigned long long id = 0;
    int rc;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);  // current_context_id's function pointers
        rc = current_context_id(&id, err);
    }
    if (rc) return rc;
    if (!id) {  // no context yet: make the device's primary context current
        *err = cudaFree(nullptr);
        if (*err != cudaSuccess) return RHG_ERR_CUDA;
        std::lock_guard<std::mutex> lk(g_static_mu);
        rc = current_context_id(&id, err);
        if (rc) return rc;
        if (!id) {
            *err = cudaErrorDeviceUninitialized;
            return RHG_ERR_CUDA;
        }
    }
    int slot = -1;
    for (int j = 0; j < kMaxContexts; ++j)
        if (g_copy_ctx[j] == id) {
            *out = &g_copy[j];
            return RHG_OK;
        } else if (slot < 0 && g_copy_ctx[j] == 0) {
            slot = j;
        }
    if (slot < 0) {  // every slot taken: no overlapped copy for this context
        *out = nullptr;
        return RHG_OK;
    }
    if (!g_phase_words_registered) {
        *err = cudaHostRegister(g_phase_words, sizeof(g_phase_words), cudaHostRegisterPortable | cudaHostRegisterMapped);
        if (*err != cudaSuccess) return RHG_ERR_CUDA;
        g_phase_words_registered = true;
    }
    HostCopy &h = g_copy[slot];
    *err = cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking);
    for (int p = 0; p < kMaxPhases && *err == cudaSuccess; ++p)
        *err = cudaEventCreateWithFlags(&h.ev[p], cudaEventDisableTiming);
    void *dm = nullptr;
    if (*err == cudaSuccess) *err = cudaHostGetDevicePointer(&dm, g_phase_words[slot], 0);
    if (*err != cudaSuccess) return RHG_ERR_CUDA;
    h.h_m = g_phase_words[slot];
    h.d_m = static_cast<uint64_t *>(dm);
    g_copy_ctx[slot] = id;
    *out = &h;
    return RHG_OK;
}

// The layout a plan describes; false if the plan is not one rhg_batch_prepare made.
bool plan_layout(const rhg_batch_plan *plan, BatchLayout &L)
{
    if (!plan || plan->count == 0 || plan->count > kMaxBatch || plan->num_tiles < plan->count ||
        plan->points >= 0xFFFFFFFFull || plan->index_entries >= 0xFFFFFFFFull || plan->verify > 1 ||
        plan->chunk_extra > kMaxListEntries)
        return false;
    L = batch_layout(plan->count, plan->points, plan->num_tiles, plan->index_entries, plan->chunk_extra);
    return L.total == plan->workspace_bytes;
}
}  // namespace
}  // namespace rhg

using namespace rhg;

// rhg_sort_keys on validated arguments: the bucket tables go to the workspace's
// Meta block, then count, scan, scatter and the per-bucket sort; *err = the
// device's error word.
Status sort_keys(const uint64_t *d_keys, uint64_t n, uint32_t num_bands, const uint32_t *bucket_bits, void *d_ws,
                 uint64_t *d_sorted_keys, uint32_t *d_sorted_ids, cudaStream_t s, uint32_t *err)
{
    Status st;
    Meta h{};
    h.B = num_bands;
    uint32_t off = 0;
    for (uint32_t j = 0; j < num_bands; ++j) {
        h.bk_off[j] = off;
        h.bk_bits[j] = bucket_bits[j];
        off += 1u << bucket_bits[j];
    }
    h.bk_off[num_bands] = off;
    h.nbuckets = off;
    char *w = static_cast<char *>(d_ws);
    const size_t o_counts = align_up(sizeof(Meta)), o_start = o_counts + align_up(uint64_t{off} * 4),
                 o_comp = o_start + align_up((uint64_t{off} + 1) * 4), o_scratch = o_comp + align_up(n * 8);
    BucketArgs ba{};
    ba.M = reinterpret_cast<Meta *>(w);
    ba.n = n;
    ba.counts = reinterpret_cast<uint32_t *>(w + o_counts);
    ba.start = reinterpret_cast<uint32_t *>(w + o_start);
    ba.comp = reinterpret_cast<uint64_t *>(w + o_comp);
    ba.scratch = reinterpret_cast<uint64_t *>(w + o_scratch);
    ba.out_keys = d_sorted_keys;
    ba.out_ids = d_sorted_ids;
    RHG_CUDA_TRY(cudaMemcpyAsync(ba.M, &h, sizeof(Meta), cudaMemcpyHostToDevice, s));
    RHG_CUDA_TRY(cudaMemsetAsync(ba.counts, 0, uint64_t{off} * 4, s));
    st = launch_bucket_count(ba, d_keys, s);
    if (!st.code) st = launch_bucket_scan(ba, s);
    if (!st.code) st = launch_bucket_scatter(ba, d_keys, s);
    if (!st.code) st = launch_bucket_sort(ba, false, s);
    if (st.code) return st;
    RHG_CUDA_TRY(cudaMemcpyAsync(err, &ba.M->error, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    RHG_CUDA_TRY(cudaStreamSynchronize(s));
    return st;
}

// Query phases for the overlapped host copy: one per ~2^23 expected edges (64 MB
// of pairs), at most 8.
uint32_t copy_phases(const rhg_params &p)
{
    const double m = static_cast<double>(p.n) * p.k * 0.5;
    const double ph = std::floor(m / 8388608.0);
    return ph < 1.0 ? 1u : (ph > 8.0 ? 8u : static_cast<uint32_t>(ph));
}

// rhg_generate_pairs_host into pinned memory: the point pipeline, then the range
// query in phases; after phase p the host copies the edges the phase added on the
// copy stream (the copy engines run beside the next phases).  A recheck list that
// overflows (rerun in FP64 mode) falls back to generate-then-copy.
int generate_host_overlapped(const rhg_params *p, void *d_ws, size_t ws_bytes, uint32_t *d_pairs, uint64_t capacity,
                             uint32_t *h_pairs, uint64_t h_capacity, HostCopy &hc, cudaStream_t stream,
                             rhg_result *res)
{
    std::memset(res, 0, sizeof(*res));
    uint32_t B;
    double ratio;
    int rc = check_params(p, &B, &ratio);
    if (rc) return rc;
    if (!d_ws) return RHG_ERR_INVALID_ARG;
    if (capacity && (!d_pairs || (reinterpret_cast<uintptr_t>(d_pairs) & 7))) return RHG_ERR_INVALID_ARG;
    const Layout L = make_layout(p->n, 0, chunk_extra(*p));
    if (ws_bytes < L.total) return RHG_ERR_OOM;
    if (reinterpret_cast<uintptr_t>(d_ws) & 255) return RHG_ERR_INVALID_ARG;
    Pipeline pl{d_ws, L, p->n};
    const PlanArgs pa = with_mapping(PlanArgs{p->n, p->k, p->alpha, p->seed, B, ratio, p->R_override,
                                              (p->flags & RHG_FLAG_FP64_ONLY) ? 0u : 1u,
                                              (p->flags & RHG_FLAG_VERIFY) ? 1u : 0u},
                                     *p);
    std::lock_guard<std::mutex> lock(hc.mu);
    SortedPoints P;
    Status st = enqueue_points(pl, pa, nullptr, nullptr, &P, stream);
    if (st.code) return finish(st, res);
    QueryArgs q{};
    q.M = pl.meta();
    q.P = P;
    q.pairs = d_pairs;
    q.capacity = capacity;
    q.heavy = at<uint4>(pl.ws, pl.L.heavy);
    q.heavy_cap = pl.L.heavy_cap;
    q.recheck = at<uint2>(pl.ws, pl.L.recheck);
    q.recheck_cap = pl.L.recheck_cap;
    q.heavy_min = kHeavyMin;
    q.bidx = at<uint32_t>(pl.ws, pl.L.bidx);
    q.verify = pa.verify != 0;
    const uint32_t phases = copy_phases(*p);
    for (uint32_t i = 0; i < phases; ++i) hc.h_m[i] = ~uint64_t{0};
    mark(RHG_STAGE_QUERY, false, stream);
    st = launch_query_phased(q, phases, hc.d_m, hc.ev, stream);
    if (st.code) return finish(st, res);
    mark(RHG_STAGE_QUERY, true, stream);
    const uint64_t limit = capacity < h_capacity ? capacity : h_capacity;
    uint64_t done = 0;
    for (uint32_t i = 0; i < phases; ++i) {
        RHG_RESULT_TRY(cudaEventSynchronize(hc.ev[i]), res);
        uint64_t m = *reinterpret_cast<volatile uint64_t *>(hc.h_m + i);
        if (m > limit) m = limit;
        if (m > done) {
            RHG_RESULT_TRY(cudaMemcpyAsync(h_pairs + 2 * done, d_pairs + 2 * done, (m - done) * 8,
                                           cudaMemcpyDeviceToHost, hc.copy),
                           res);
            done = m;
        }
    }
    Meta h;
    st = read_meta(pl.meta(), &h, stream);
    if (st.code) return finish(st, res);
    RHG_RESULT_TRY(cudaStreamSynchronize(hc.copy), res);
    if (h.error == kErrListFull && h.filter) {  // the FP64 rerun, then one copy
        PlanArgs p64 = pa;
        p64.allow_filter = 0;
        st = run_pipeline(pl, p64, nullptr, nullptr, Output::Pairs, d_pairs, capacity, &h, stream);
        if (st.code) return finish(st, res);
        fill_result(res, h);
        if (h.error) return error_from_meta(h.error);
        if (h.m > capacity || h.m > h_capacity) return RHG_ERR_OVERFLOW;
        if (h.m) RHG_RESULT_TRY(cudaMemcpyAsync(h_pairs, d_pairs, h.m * 8, cudaMemcpyDeviceToHost, stream), res);
        RHG_RESULT_TRY(cudaStreamSynchronize(stream), res);
        return RHG_OK;
    }
    fill_result(res, h);
    if (h.error) return error_from_meta(h.error);
    if (h.m > capacity || h.m > h_capacity) return RHG_ERR_OVERFLOW;
    return RHG_OK;
}

extern "C" {

const char *rhg_status_str(int status)
{
    switch (status) {
        case RHG_OK: return "RHG_OK";
        case RHG_ERR_INVALID_ARG: return "RHG_ERR_INVALID_ARG";
        case RHG_ERR_NO_SOLUTION: return "RHG_ERR_NO_SOLUTION";
        case RHG_ERR_OOM: return "RHG_ERR_OOM";
        case RHG_ERR_CUDA: return "RHG_ERR_CUDA";
        case RHG_ERR_TIMEOUT: return "RHG_ERR_TIMEOUT";
        case RHG_ERR_OVERFLOW: return "RHG_ERR_OVERFLOW";
        default: return "RHG_ERR_UNKNOWN";
    }
}

int rhg_version(void) { return 4; }

int rhg_set_stage_events(void *const *events, uint32_t count)
{
    g_events = count ? events : nullptr;
    g_num_events = events ? count : 0;
    return RHG_OK;
}

uint64_t rhg_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

uint32_t rhg_default_bands(uint64_t n) { return default_bands(n); }

int rhg_workspace_bytes(const rhg_params *p, uint64_t capacity_entries, size_t *bytes)
{
    uint32_t B;
    double ratio;
    const int rc = check_params(p, &B, &ratio);
    if (rc) return rc;
    if (!bytes) return RHG_ERR_INVALID_ARG;
    *bytes = make_layout(p->n, capacity_entries, chunk_extra(*p)).total;
    return RHG_OK;
}

int rhg_workspace_bytes_points(uint64_t n, uint32_t num_bands, size_t *bytes)
{
    if (!bytes || n < 1 || n > 0xFFFFFFFFull || num_bands > RHG_MAX_BANDS) return RHG_ERR_INVALID_ARG;
    *bytes = make_layout(n, 0).total;
    return RHG_OK;
}

size_t rhg_plan_workspace_bytes(void) { return align_up(sizeof(Meta)); }

int rhg_plan(const rhg_params *p, void *d_workspace, size_t workspace_bytes, void *stream, double *R_out,
             double *h_c, uint32_t *num_bands_out)
{
    uint32_t B;
    double ratio;
    const int rc = check_params(p, &B, &ratio);
    if (rc) return rc;
    if (!R_out || !h_c || !num_bands_out || !d_workspace) return RHG_ERR_INVALID_ARG;
    if (workspace_bytes < sizeof(Meta)) return RHG_ERR_OOM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Meta *d = static_cast<Meta *>(d_workspace);
    const PlanArgs pa = with_mapping(PlanArgs{p->n, p->k, p->alpha, p->seed, B, ratio, p->R_override, 1u, 0u}, *p);
    const Status st = launch_plan(d, pa, s);
    if (st.code) return st.code;
    Meta h;
    if (cudaMemcpyAsync(&h, d, sizeof(Meta), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RHG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RHG_ERR_CUDA;
    if (h.error) return error_from_meta(h.error);
    *R_out = h.R;
    *num_bands_out = h.B;
    for (uint32_t j = 0; j <= h.B; ++j) h_c[j] = h.c[j];
    return RHG_OK;
}

int rhg_target_radius(uint64_t n, double k, double alpha, void *d_workspace, size_t workspace_bytes,
                      void *stream, double *R_out)
{
    if (!R_out) return RHG_ERR_INVALID_ARG;
    rhg_params p{};
    p.n = n;
    p.k = k;
    p.alpha = alpha;
    double c[RHG_MAX_BANDS + 1];
    uint32_t B = 0;
    return rhg_plan(&p, d_workspace, workspace_bytes, stream, R_out, c, &B);
}

int rhg_sample_points(const rhg_params *p, void *d_workspace, size_t workspace_bytes, double *d_phi,
                      double *d_r, void *stream, double *R_out)
{
    uint32_t B;
    double ratio;
    const int rc = check_params(p, &B, &ratio);
    if (rc) return rc;
    if (!d_workspace || !d_phi || !d_r) return RHG_ERR_INVALID_ARG;
    if (workspace_bytes < sizeof(Meta)) return RHG_ERR_OOM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Meta *M = static_cast<Meta *>(d_workspace);
    const PlanArgs pa = with_mapping(PlanArgs{p->n, p->k, p->alpha, p->seed, B, ratio, p->R_override, 1u, 0u}, *p);
    Status st = launch_plan(M, pa, s);
    if (st.code) return st.code;
    st = launch_points_by_id(M, p->n, p->seed, d_phi, d_r, s);
    if (st.code) return st.code;
    Meta h;
    if (cudaMemcpyAsync(&h, M, sizeof(Meta), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RHG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RHG_ERR_CUDA;
    if (h.error) return error_from_meta(h.error);
    if (R_out) *R_out = h.R;
    return RHG_OK;
}

int rhg_generate_pairs(const rhg_params *p, void *d_workspace, size_t workspace_bytes, uint32_t *d_pairs,
                       uint64_t capacity_edges, void *stream, rhg_result *result)
{
    return generate(p, d_workspace, workspace_bytes, Output::Pairs, d_pairs, capacity_edges, nullptr, nullptr,
                    static_cast<cudaStream_t>(stream), result);
}

int rhg_generate_pairs_host(const rhg_params *p, void *d_workspace, size_t workspace_bytes, uint32_t *d_pairs,
                            uint64_t capacity_edges, uint32_t *h_pairs, uint64_t h_capacity_edges, void *stream,
                            rhg_result *result)
{
    if (!h_pairs && h_capacity_edges) return RHG_ERR_INVALID_ARG;
    rhg_result local{};
    rhg_result *res = result ? result : &local;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // pinned host memory the copy engines reach directly: the copy of each query
    // phase's edges overlaps the later phases
    cudaPointerAttributes attr{};
    const bool pinned = h_pairs && cudaPointerGetAttributes(&attr, h_pairs) == cudaSuccess &&
                        attr.type == cudaMemoryTypeHost;
    cudaGetLastError();  // a pageable pointer may leave an error behind
    if (pinned) {
        HostCopy *hc = nullptr;
        cudaError_t err = cudaSuccess;
        int rc = host_copy_resources(&hc, &err);
        if (rc) {
            std::memset(res, 0, sizeof(*res));
            res->cuda_error = err;
            return rc;
        }
        if (hc) return generate_host_overlapped(p, d_workspace, workspace_bytes, d_pairs, capacity_edges, h_pairs,
                                                h_capacity_edges, *hc, s, res);
    }
    const int rc = rhg_generate_pairs(p, d_workspace, workspace_bytes, d_pairs, capacity_edges, stream, res);
    if (rc) return rc;
    if (res->m > h_capacity_edges) return RHG_ERR_OVERFLOW;
    if (res->m) {
        const cudaError_t e =
            cudaMemcpyAsync(h_pairs, d_pairs, res->m * 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
            res->cuda_error = e;
            return RHG_ERR_CUDA;
        }
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        res->cuda_error = e;
        return RHG_ERR_CUDA;
    }
    return RHG_OK;
}

int rhg_generate_csr(const rhg_params *p, void *d_workspace, size_t workspace_bytes, uint64_t *d_row_ptr,
                     uint32_t *d_col, uint64_t capacity_entries, void *stream, rhg_result *result)
{
    return generate(p, d_workspace, workspace_bytes, Output::Csr, nullptr, capacity_entries, d_row_ptr, d_col,
                    static_cast<cudaStream_t>(stream), result);
}

int rhg_edges_from_points(const double *d_phi, const double *d_r, uint64_t n, double R, uint32_t num_bands,
                          double band_ratio, uint32_t flags, void *d_workspace, size_t workspace_bytes,
                          uint32_t *d_pairs, uint64_t capacity_edges, void *stream, rhg_result *result)
{
    if (result) std::memset(result, 0, sizeof(*result));
    if (n < 1 || n > 0xFFFFFFFFull || !d_phi || !d_r || !d_workspace) return RHG_ERR_INVALID_ARG;
    if (!(R > 0.0) || !(R <= 700.0) || num_bands > RHG_MAX_BANDS) return RHG_ERR_INVALID_ARG;
    if (band_ratio < 0.0 || !std::isfinite(band_ratio) || (flags & ~kKnownFlags)) return RHG_ERR_INVALID_ARG;
    if (capacity_edges && (!d_pairs || (reinterpret_cast<uintptr_t>(d_pairs) & 7))) return RHG_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_workspace) & 255) return RHG_ERR_INVALID_ARG;
    const uint32_t B = num_bands ? num_bands : default_bands(n < 2 ? 2 : n);
    const double ratio = band_ratio > 0.0 ? band_ratio : 0.9;
    const Layout L = make_layout(n, 0);
    if (workspace_bytes < L.total) return RHG_ERR_OOM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Pipeline pl{d_workspace, L, n};
    // alpha and k only enter the sampler and the R solve, which are not used here
    const PlanArgs pa = with_mapping(PlanArgs{n, 1.0, 1.0, 0, B, ratio, R, (flags & RHG_FLAG_FP64_ONLY) ? 0u : 1u,
                                              (flags & RHG_FLAG_VERIFY) ? 1u : 0u},
                                     0, 0, 0);
    Meta h;
    const Status st = run_pipeline(pl, pa, d_phi, d_r, Output::Pairs, d_pairs, capacity_edges, &h, s);
    if (st.code) return finish(st, result);
    fill_result(result, h);
    if (h.error) return error_from_meta(h.error);
    if (h.m > capacity_edges) return RHG_ERR_OVERFLOW;
    return RHG_OK;
}

int rhg_generate_pairs_static(const rhg_params *p, uint32_t *d_pairs, uint64_t capacity_edges, void *stream,
                              rhg_result *result)
{
    if (result) std::memset(result, 0, sizeof(*result));
    if (!p || p->n > RHG_STATIC_MAX_POINTS) return RHG_ERR_INVALID_ARG;
    const size_t need = make_layout(p->n, 0, chunk_extra(*p)).total;
    if (need > RHG_STATIC_SCRATCH_BYTES) return RHG_ERR_INVALID_ARG;
    void *ws = nullptr;
    cudaError_t err = cudaSuccess;
    const int rc = static_scratch(&ws, &err);
    if (rc) {
        if (result) result->cuda_error = static_cast<int32_t>(err);
        return rc;
    }
    return generate(p, ws, RHG_STATIC_SCRATCH_BYTES, Output::Pairs, d_pairs, capacity_edges, nullptr, nullptr,
                    static_cast<cudaStream_t>(stream), result);
}

int rhg_batch_workspace_bytes(const rhg_params *graphs, uint32_t count, size_t *bytes)
{
    if (!bytes) return RHG_ERR_INVALID_ARG;
    BatchHost h;
    const int rc = batch_host(graphs, count, nullptr, h);
    if (rc) return rc;
    *bytes = batch_layout(h).total;
    return RHG_OK;
}

int rhg_generate_batch(const rhg_params *graphs, uint32_t count, void *d_workspace, size_t workspace_bytes,
                       uint32_t *d_pairs, const uint64_t *pair_offsets, void *stream, rhg_batch_graph *results,
                       rhg_result *totals)
{
    if (totals) std::memset(totals, 0, sizeof(*totals));
    if (!d_workspace || !pair_offsets || !results) return RHG_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_workspace) & 255) return RHG_ERR_INVALID_ARG;
    BatchHost h;
    int rc = batch_host(graphs, count, pair_offsets, h);
    if (rc) return rc;
    if (h.out_off[count] && (!d_pairs || (reinterpret_cast<uintptr_t>(d_pairs) & 7))) return RHG_ERR_INVALID_ARG;
    const BatchLayout L = batch_layout(h);
    if (workspace_bytes < L.total) return RHG_ERR_OOM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<uint4> res(2 * static_cast<size_t>(count));
    Meta ctl;
    for (int attempt = 0; attempt < 2; ++attempt) {
        Status st = upload_tables(d_workspace, L, h, s);
        if (st.code) return finish(st, totals);
        st = enqueue_batch(d_workspace, L, h.G, h.N, h.tiles.size(), any_verify(h), d_pairs, s);
        if (st.code) return finish(st, totals);
        const cudaError_t e1 = cudaMemcpyAsync(res.data(), at<uint4>(d_workspace, L.results),
                                               res.size() * sizeof(uint4), cudaMemcpyDeviceToHost, s);
        const cudaError_t e2 = cudaMemcpyAsync(&ctl, at<Meta>(d_workspace, L.metas) + count, sizeof(Meta),
                                               cudaMemcpyDeviceToHost, s);
        const cudaError_t e3 = cudaStreamSynchronize(s);
        const cudaError_t e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
        if (e != cudaSuccess) {
            if (totals) totals->cuda_error = static_cast<int32_t>(e);
            return RHG_ERR_CUDA;
        }
        if (ctl.error != kErrListFull || attempt) break;
        for (auto &a : h.args) a.allow_filter = 0;  // the FP64 mode needs no recheck list
    }
    return fill_batch_results(count, res.data(), ctl, h.out_off.data(), results, totals);
}

int rhg_batch_prepare(const rhg_params *graphs, uint32_t count, const uint64_t *pair_offsets, void *d_workspace,
                      size_t workspace_bytes, void *stream, rhg_batch_plan *plan)
{
    if (plan) std::memset(plan, 0, sizeof(*plan));
    if (!d_workspace || !pair_offsets || !plan) return RHG_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_workspace) & 255) return RHG_ERR_INVALID_ARG;
    BatchHost h;
    const int rc = batch_host(graphs, count, pair_offsets, h);
    if (rc) return rc;
    const BatchLayout L = batch_layout(h);
    if (workspace_bytes < L.total) return RHG_ERR_OOM;
    const Status st = upload_tables(d_workspace, L, h, static_cast<cudaStream_t>(stream));
    if (st.code) return st.code;
    plan->count = count;
    plan->verify = any_verify(h) ? 1u : 0u;
    plan->num_tiles = h.tiles.size();
    plan->points = h.N;
    plan->index_entries = h.idx_total;
    plan->pair_capacity = h.out_off[count];
    plan->workspace_bytes = L.total;
    plan->chunk_extra = h.chunk_extra;
    return RHG_OK;
}

int rhg_batch_launch(const rhg_batch_plan *plan, void *d_workspace, uint32_t *d_pairs, void *stream)
{
    BatchLayout L;
    if (!plan_layout(plan, L) || !d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
        return RHG_ERR_INVALID_ARG;
    if (plan->pair_capacity && (!d_pairs || (reinterpret_cast<uintptr_t>(d_pairs) & 7))) return RHG_ERR_INVALID_ARG;
    const Status st = enqueue_batch(d_workspace, L, plan->count, plan->points, plan->num_tiles, plan->verify != 0,
                                    d_pairs, static_cast<cudaStream_t>(stream));
    return st.code;
}

int rhg_batch_read_results(const rhg_batch_plan *plan, const void *d_workspace, void *stream,
                           rhg_batch_graph *results, rhg_result *totals)
{
    if (totals) std::memset(totals, 0, sizeof(*totals));
    BatchLayout L;
    if (!plan_layout(plan, L) || !d_workspace || !results) return RHG_ERR_INVALID_ARG;
    const uint32_t count = plan->count;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<uint4> res(2 * static_cast<size_t>(count));
    std::vector<uint64_t> out_off(static_cast<size_t>(count) + 1);
    Meta ctl;
    const char *ws = static_cast<const char *>(d_workspace);
    const cudaError_t e1 =
        cudaMemcpyAsync(res.data(), ws + L.results, res.size() * sizeof(uint4), cudaMemcpyDeviceToHost, s);
    const cudaError_t e2 = cudaMemcpyAsync(&ctl, ws + L.metas + count * sizeof(Meta), sizeof(Meta),
                                           cudaMemcpyDeviceToHost, s);
    const cudaError_t e3 =
        cudaMemcpyAsync(out_off.data(), ws + L.out_off, out_off.size() * 8, cudaMemcpyDeviceToHost, s);
    const cudaError_t e4 = cudaStreamSynchronize(s);
    const cudaError_t e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3 != cudaSuccess ? e3 : e4;
    if (e != cudaSuccess) {
        if (totals) totals->cuda_error = static_cast<int32_t>(e);
        return RHG_ERR_CUDA;
    }
    return fill_batch_results(count, res.data(), ctl, out_off.data(), results, totals);
}

int rhg_batch_stage_times(const rhg_batch_plan *plan, const void *d_workspace, void *stream, double *ms,
                          uint32_t count)
{
    BatchLayout L;
    if (!plan_layout(plan, L) || !d_workspace || !ms || count < RHG_BATCH_STAGE_COUNT) return RHG_ERR_INVALID_ARG;
    static_assert(RHG_BATCH_STAGE_COUNT + 1 == kBatchStages, "one duration between consecutive stage marks");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Meta ctl;
    const char *ws = static_cast<const char *>(d_workspace);
    if (cudaMemcpyAsync(&ctl, ws + L.metas + plan->count * sizeof(Meta), sizeof(Meta), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return RHG_ERR_CUDA;
    for (uint32_t k = 0; k < RHG_BATCH_STAGE_COUNT; ++k)
        ms[k] = ctl.stage_ns[k + 1] > ctl.stage_ns[k] ? 1e-6 * static_cast<double>(ctl.stage_ns[k + 1] - ctl.stage_ns[k])
                                                       : 0.0;
    return RHG_OK;
}

int rhg_grid_barrier_test(uint32_t missing, uint64_t timeout_ns, void *d_workspace, size_t workspace_bytes,
                          void *stream)
{
    if (!d_workspace || missing > 1024 || timeout_ns == 0 || timeout_ns > 10ull * 1000 * 1000 * 1000)
        return RHG_ERR_INVALID_ARG;
    if (workspace_bytes < align_up(sizeof(Meta)) + 256) return RHG_ERR_OOM;
    if (reinterpret_cast<uintptr_t>(d_workspace) & 255) return RHG_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Meta *M = static_cast<Meta *>(d_workspace);
    uint32_t *bar = at<uint32_t>(d_workspace, align_up(sizeof(Meta)));
    if (cudaMemsetAsync(M, 0, sizeof(Meta), s) != cudaSuccess) return RHG_ERR_CUDA;
    const Status st = launch_barrier_test(M, bar, missing, timeout_ns, s);
    if (st.code) return st.code;
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, &M->error, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return RHG_ERR_CUDA;
    return error_from_meta(err);
}

int rhg_draw_movement(uint64_t n, uint64_t seed, double phi_lo, double phi_hi, double r_lo, double r_hi,
                      double *d_tau_phi, double *d_tau_r, void *stream)
{
    if (n && (!d_tau_phi || !d_tau_r)) return RHG_ERR_INVALID_ARG;
    if (!std::isfinite(phi_lo) || !std::isfinite(phi_hi) || !std::isfinite(r_lo) || !std::isfinite(r_hi) ||
        phi_hi < phi_lo || r_hi < r_lo)
        return RHG_ERR_INVALID_ARG;
    return launch_draw_movement(n, seed, phi_lo, phi_hi, r_lo, r_hi, d_tau_phi, d_tau_r,
                                static_cast<cudaStream_t>(stream))
        .code;
}

int rhg_move_points(const uint32_t *d_ids, uint64_t count, uint64_t n, double *d_phi, double *d_r,
                    const double *d_tau_phi, double *d_tau_r, double R, double alpha, void *stream)
{
    if (count && (!d_ids || !d_phi || !d_r || !d_tau_phi || !d_tau_r)) return RHG_ERR_INVALID_ARG;
    if (count > n || n > 0xFFFFFFFFull) return RHG_ERR_INVALID_ARG;
    if (!(R > 0.0) || !(R <= 700.0) || !(alpha > 0.5) || !(alpha <= 100.0) || alpha * R > 700.0)
        return RHG_ERR_INVALID_ARG;
    return launch_move(d_ids, count, n, d_phi, d_r, d_tau_phi, d_tau_r, R, alpha, static_cast<cudaStream_t>(stream))
        .code;
}

int rhg_workspace_bytes_update(uint64_t n, uint64_t moved_count, uint32_t num_bands, size_t *bytes)
{
    if (!bytes || n < 1 || n > 0xFFFFFFFFull || moved_count > n || num_bands > RHG_MAX_BANDS)
        return RHG_ERR_INVALID_ARG;
    *bytes = update_layout(n, moved_count, num_bands ? num_bands : default_bands(n < 2 ? 2 : n)).total;
    return RHG_OK;
}

int rhg_update_edges(const double *d_phi, const double *d_r, uint64_t n, double R, uint32_t num_bands,
                     double band_ratio, uint32_t flags, const uint32_t *d_moved_ids, uint64_t moved_count,
                     const uint32_t *d_old_pairs, uint64_t m_old, void *d_workspace, size_t workspace_bytes,
                     uint32_t *d_new_pairs, uint64_t capacity_edges, void *stream, rhg_result *result)
{
    if (result) std::memset(result, 0, sizeof(*result));
    if (n < 1 || n > 0xFFFFFFFFull || !d_phi || !d_r || !d_workspace) return RHG_ERR_INVALID_ARG;
    if (!(R > 0.0) || !(R <= 700.0) || num_bands > RHG_MAX_BANDS) return RHG_ERR_INVALID_ARG;
    if (band_ratio < 0.0 || !std::isfinite(band_ratio) || (flags & ~RHG_FLAG_FP64_ONLY)) return RHG_ERR_INVALID_ARG;
    if (moved_count > n || (moved_count && !d_moved_ids) || (m_old && !d_old_pairs)) return RHG_ERR_INVALID_ARG;
    if (capacity_edges && (!d_new_pairs || (reinterpret_cast<uintptr_t>(d_new_pairs) & 7))) return RHG_ERR_INVALID_ARG;
    if (m_old && (reinterpret_cast<uintptr_t>(d_old_pairs) & 7)) return RHG_ERR_INVALID_ARG;
    if (m_old && capacity_edges && d_new_pairs == d_old_pairs) return RHG_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_workspace) & 255) return RHG_ERR_INVALID_ARG;
    const uint32_t B = num_bands ? num_bands : default_bands(n < 2 ? 2 : n);
    const UpdateLayout U = update_layout(n, moved_count, B);
    if (workspace_bytes < U.total) return RHG_ERR_OOM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double ratio = band_ratio > 0.0 ? band_ratio : 0.9;
    const PlanArgs pa =
        with_mapping(PlanArgs{n, 1.0, 1.0, 0, B, ratio, R, (flags & RHG_FLAG_FP64_ONLY) ? 0u : 1u, 0u}, 0, 0, 0);
    Pipeline pl{d_workspace, U.L, n};
    Meta *M = pl.meta();
    SortedPoints P;
    Status st = enqueue_points(pl, pa, d_phi, d_r, &P, s);
    if (st.code) return finish(st, result);
    QueryArgs q{};
    q.M = M;
    q.P = P;
    q.src_phi = d_phi;
    q.src_r = d_r;
    q.pairs = d_new_pairs;
    q.capacity = capacity_edges;
    q.bidx = at<uint32_t>(d_workspace, U.L.bidx);
    uint8_t *moved_id = at<uint8_t>(d_workspace, U.moved_id), *moved_pos = at<uint8_t>(d_workspace, U.moved_pos);
    uint32_t *owners = at<uint32_t>(d_workspace, U.owners), *counts = at<uint32_t>(d_workspace, U.counts);
    uint64_t *offsets = at<uint64_t>(d_workspace, U.offsets);
    // the plan zeroed these counters: work_counter lists the moved vertices, m the
    // kept edges, and heavy_n with heavy_next (one 64-bit word) the chunks
    unsigned long long *owner_n = reinterpret_cast<unsigned long long *>(&M->work_counter);
    unsigned long long *kept = reinterpret_cast<unsigned long long *>(&M->m);
    unsigned long long *chunk_n = reinterpret_cast<unsigned long long *>(&M->heavy_n);
    static_assert(offsetof(Meta, heavy_next) == offsetof(Meta, heavy_n) + 4 && offsetof(Meta, heavy_n) % 8 == 0,
                  "heavy_n and heavy_next form one aligned 64-bit word");
    uint4 *chunks = at<uint4>(d_workspace, U.chunks);
    const uint64_t slots = moved_count * B + U.chunk_cap;
    mark(RHG_STAGE_QUERY, false, s);
    if (!st.code) st = launch_bucket_index(q, s);
    uint32_t *moved_bits = at<uint32_t>(d_workspace, U.moved_bits);
    if (!st.code) st = launch_mark_moved(d_moved_ids, moved_count, n, moved_id, moved_bits, s);
    if (!st.code) st = launch_owners(M, P.id, n, moved_id, moved_pos, owners, moved_count, owner_n, s);
    if (!st.code)
        st = launch_subset_query(q, owners, moved_count, owner_n, chunks, U.chunk_cap, chunk_n, moved_pos, counts,
                                 nullptr, nullptr, 0, false, s);
    if (!st.code) st = launch_scan(counts, slots, offsets, at<void>(d_workspace, U.scan_tmp), s);
    if (!st.code) st = launch_keep_old(d_old_pairs, m_old, moved_bits, n, d_new_pairs, capacity_edges, kept, s);
    if (!st.code)
        st = launch_subset_query(q, owners, moved_count, owner_n, chunks, U.chunk_cap, chunk_n, moved_pos, counts,
                                 offsets, kept, capacity_edges, true, s);
    if (!st.code) st = launch_add_total(kept, offsets + slots, s);
    if (st.code) return finish(st, result);
    mark(RHG_STAGE_QUERY, true, s);
    Meta h;
    st = read_meta(M, &h, s);
    if (st.code) return finish(st, result);
    fill_result(result, h);
    if (h.error) return error_from_meta(h.error);
    if (h.work_counter != moved_count) return RHG_ERR_INVALID_ARG;  // an id repeated or out of range
    if (h.m > capacity_edges) return RHG_ERR_OVERFLOW;
    return RHG_OK;
}

int rhg_sort_keys_workspace_bytes(uint64_t n, uint32_t num_bands, const uint32_t *bucket_bits, size_t *bytes)
{
    if (!bytes || !bucket_bits || num_bands < 1 || num_bands > static_cast<uint32_t>(kMaxBands) ||
        n > 0xFFFFFFFFull)
        return RHG_ERR_INVALID_ARG;
    uint64_t nb = 0;
    for (uint32_t j = 0; j < num_bands; ++j) {
        if (bucket_bits[j] > 24) return RHG_ERR_INVALID_ARG;
        nb += uint64_t{1} << bucket_bits[j];
    }
    if (nb > 0xFFFFFFFEull) return RHG_ERR_INVALID_ARG;
    *bytes = align_up(sizeof(Meta)) + align_up(nb * 4) + align_up((nb + 1) * 4) + 2 * align_up(n * 8);
    return RHG_OK;
}

int rhg_sort_keys(const uint64_t *d_keys, uint64_t n, uint32_t num_bands, const uint32_t *bucket_bits,
                  void *d_workspace, size_t workspace_bytes, uint64_t *d_sorted_keys, uint32_t *d_sorted_ids,
                  void *stream)
{
    size_t need = 0;
    int rc = rhg_sort_keys_workspace_bytes(n, num_bands, bucket_bits, &need);
    if (rc) return rc;
    if (n && (!d_keys || !d_sorted_keys || !d_sorted_ids || !d_workspace)) return RHG_ERR_INVALID_ARG;
    if (!n) return RHG_OK;
    if (reinterpret_cast<uintptr_t>(d_workspace) & 255) return RHG_ERR_INVALID_ARG;
    if (workspace_bytes < need) return RHG_ERR_OOM;
    uint32_t err = 0;
    const Status st = sort_keys(d_keys, n, num_bands, bucket_bits, d_workspace, d_sorted_keys, d_sorted_ids,
                                static_cast<cudaStream_t>(stream), &err);
    if (st.code) return st.code;
    return err ? RHG_ERR_INVALID_ARG : RHG_OK;
}

int rhg_dm_eval(int fn, const double *d_in, double *d_out, uint64_t count, void *stream)
{
    if (fn < 0 || fn > 5 || (count && (!d_in || !d_out))) return RHG_ERR_INVALID_ARG;
    if (!count) return RHG_OK;
    const Status st = launch_dm_eval(fn, d_in, d_out, count, static_cast<cudaStream_t>(stream));
    return st.code;
}

}  // extern "C"
