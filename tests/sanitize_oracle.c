/* Drives every entry point of the oracle (oracle/rhg_oracle.c) on small inputs,
 * including capacities smaller than the output, so that a build with
 * -fsanitize=address,undefined reports any out-of-bounds access, leak or
 * undefined behaviour.  Test infrastructure: built and run by
 * tests/test_oracle_sanitizers.py.  Exit status 0 when the results agree. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

void ro_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
void ro_philox4x64_batch(uint64_t count, const uint64_t ctr0[4], const uint64_t key[2], uint64_t *out);
double ro_exp(double x);
double ro_log(double x);
double ro_cos(double d);
double ro_cosh(double x);
double ro_sinh(double x);
double ro_asinh(double y);
double ro_kbar(double R, uint64_t n, double alpha);
int ro_target_radius(uint64_t n, double k, double alpha, double *R_out);
uint32_t ro_default_bands(uint64_t n);
int ro_boundaries(double R, uint32_t B, double p, double *c);
int ro_sample_points(uint64_t n, double alpha, double R, uint64_t seed, uint64_t first, double *phi, double *r);
int ro_edge(double phv, double rv, double phw, double rw, double R);
int64_t ro_brute_edges(uint64_t n, const double *phi, const double *r, double R, uint32_t *pairs,
                       uint64_t capacity);
int64_t ro_neighbors(uint64_t v, uint64_t n, const double *phi, const double *r, double R, uint32_t *out,
                     uint64_t capacity);
int64_t ro_band_edges(uint64_t n, const double *phi, const double *r, double R, uint32_t B, double p,
                      uint32_t *pairs, uint64_t capacity, int64_t *stats);
int ro_band_assign(uint64_t n, const double *r, double R, uint32_t B, double p, uint32_t *band);
int64_t ro_band_count_subset(uint64_t n, const double *phi, const double *r, double R, uint32_t B, double p,
                             const uint32_t *ids, uint64_t nids, int32_t *threads, int64_t *stats);
void *ro_prepare(uint64_t n, const double *phi, const double *r, double R, uint32_t B, double p);
int64_t ro_prepared_count(void *handle, const uint32_t *ids, uint64_t nids, int32_t *threads, int64_t *stats);
int64_t ro_prepared_upper_pairs(void *handle, uint64_t u0, uint64_t u1, uint32_t *pairs, uint64_t capacity);
int ro_prepared_window_misses(void *handle, const uint32_t *ids, uint64_t nids, double theta_scale, int64_t *out);
void ro_prepared_free(void *handle);
void ro_draw_movement(uint64_t n, uint64_t seed, double phi_lo, double phi_hi, double r_lo, double r_hi,
                      double *tau_phi, double *tau_r);
void ro_move(uint64_t count, const uint32_t *ids, double *phi, double *r, const double *tau_phi, double *tau_r,
             double R, double alpha, int32_t coord);
void ro_constants(double *out);

static int fails = 0;
#define CHECK(c)                                                   \
    do {                                                           \
        if (!(c)) {                                                \
            fprintf(stderr, "check failed line %d: %s\n", __LINE__, #c); \
            ++fails;                                               \
        }                                                          \
    } while (0)

static void graph_case(uint64_t n, double k, double alpha, uint64_t seed)
{
    double R = 0.0;
    CHECK(ro_target_radius(n, k, alpha, &R) == 0);
    double *phi = malloc(n * sizeof(double)), *r = malloc(n * sizeof(double));
    CHECK(ro_sample_points(n, alpha, R, seed, 0, phi, r) == 0);
    int64_t m = ro_brute_edges(n, phi, r, R, NULL, 0);
    CHECK(m >= 0);
    uint32_t *pairs = malloc((size_t)(m + 1) * 2 * sizeof(uint32_t));
    CHECK(ro_brute_edges(n, phi, r, R, pairs, (uint64_t)m) == m);
    uint32_t B = ro_default_bands(n);
    for (uint32_t b = 1; b <= B + 2; b += 1 + B / 3) {
        int64_t stats[6] = {0, 0, 0, 0, 0, 0};
        CHECK(ro_band_edges(n, phi, r, R, b, 0.9, pairs, (uint64_t)m / 2, stats) == m);  /* short room */
        CHECK(ro_band_edges(n, phi, r, R, b, 0.9, pairs, (uint64_t)m, stats) == m);
    }
    uint32_t *band = malloc(n * sizeof(uint32_t)), *ids = malloc(n * sizeof(uint32_t));
    CHECK(ro_band_assign(n, r, R, B, 0.9, band) == 0);
    for (uint64_t i = 0; i < n; ++i) CHECK(band[i] < B);
    for (uint64_t i = 0; i < n; ++i) ids[i] = (uint32_t)i;
    int32_t nt = 0;
    int64_t st6[6];
    CHECK(ro_band_count_subset(n, phi, r, R, B, 0.9, ids, n, &nt, NULL) == m);
    CHECK(ro_band_count_subset(n, phi, r, R, B, 0.9, ids, n, &nt, st6) == m);
    void *h = ro_prepare(n, phi, r, R, B, 0.9);
    CHECK(h != NULL);
    if (h) {
        CHECK(ro_prepared_count(h, ids, n, &nt, NULL) == m);
        CHECK(ro_prepared_count(h, ids, n, &nt, st6) == m);
        /* ordered pairs: short room first (nothing written), then the exact room, in two ranges */
        CHECK(ro_prepared_upper_pairs(h, 0, n, pairs, (uint64_t)m / 2) == m);
        int64_t m1 = ro_prepared_upper_pairs(h, 0, n / 2, pairs, (uint64_t)m);
        CHECK(m1 >= 0 && m1 <= m);
        CHECK(ro_prepared_upper_pairs(h, n / 2, n, pairs + 2 * (m1 > 0 ? m1 : 0), (uint64_t)(m - m1)) == m - m1);
        CHECK(ro_prepared_upper_pairs(h, n, n + 1, pairs, 0) < 0);  /* range beyond n */
        int64_t wm[4];
        CHECK(ro_prepared_window_misses(h, ids, n < 50 ? n : 50, 1.0, wm) == 0 && wm[1] == 0);
        ro_prepared_free(h);
    }
    int64_t deg = 0;
    uint32_t *row = malloc(n * sizeof(uint32_t));
    for (uint64_t v = 0; v < n; v += 1 + n / 17) {
        int64_t d = ro_neighbors(v, n, phi, r, R, row, 1);  /* room for one */
        CHECK(d >= 0 && ro_neighbors(v, n, phi, r, R, row, n) == d);
        deg += d;
    }
    CHECK(deg >= 0);
    double *tp = malloc(n * sizeof(double)), *tr = malloc(n * sizeof(double));
    ro_draw_movement(n, seed, -1.0, 1.0, -10.0, 1.0, tp, tr);
    ro_move(n / 2, ids + n / 4, phi, r, tp, tr, R, alpha, 0);
    ro_move(n / 2, ids + n / 4, phi, r, tp, tr, R, alpha, 1);
    for (uint64_t i = 0; i < n; ++i) CHECK(phi[i] >= 0.0 && r[i] >= 0.0 && r[i] <= R);
    free(tp);
    free(tr);
    free(row);
    free(band);
    free(ids);
    free(pairs);
    free(phi);
    free(r);
}

int main(void)
{
    uint64_t ctr[4] = {1, 2, 3, 4}, key[2] = {5, 6}, out[4], batch[4 * 9];
    ro_philox4x64(ctr, key, out);
    ro_philox4x64_batch(9, ctr, key, batch);
    CHECK(batch[0] == out[0] && batch[3] == out[3]);
    for (double x = -700.0; x <= 700.0; x += 0.37) {
        CHECK(ro_exp(x) > 0.0);
        CHECK(ro_cosh(x / 20.0) >= 1.0);
        (void)ro_sinh(x / 20.0);
        (void)ro_cos(x);
        if (x > 0) CHECK(ro_log(x) == ro_log(x));
        CHECK(ro_asinh(x) == ro_asinh(x));
    }
    double c[70], consts[10];
    ro_constants(consts);
    CHECK(ro_boundaries(20.0, 64, 0.9, c) == 0);
    CHECK(ro_boundaries(20.0, 65, 0.9, c) != 0);
    CHECK(ro_kbar(20.0, 1000, 1.0) > 0.0);
    double R;
    CHECK(ro_target_radius(100, 1e9, 1.0, &R) != 0);  /* unreachable degree */
    CHECK(ro_edge(0.0, 1.0, 0.0, 1.0, 5.0) == 1);
    graph_case(2, 0.5, 1.0, 1);
    graph_case(300, 6.0, 1.0, 2);
    graph_case(1500, 20.0, 0.6, 3);
    graph_case(800, 3.0, 3.0, 4);
    if (fails) fprintf(stderr, "%d checks failed\n", fails);
    return fails ? 1 : 0;
}
