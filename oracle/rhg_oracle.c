/*
 * rhg_oracle.c -- plain, slow CPU oracle for threshold random hyperbolic graphs
 * (von Looz, Ozdayi, Laue, Meyerhenke, "Generating massive complex networks with
 * hyperbolic geometry faster in practice", arXiv:1606.09481).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  It is used by tests/, by __graft_entry__.smoke() and by the
 * CPU-baseline leg of bench.py, and nowhere else.  It shares no code with the
 * CUDA path: the only common ground is the written definition of the
 * deterministic FP64 operation sequences, which both sides implement separately.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared [-fopenmp].
 * Every floating-point expression below is a sequence of separately rounded IEEE
 * binary64 operations (round to nearest even); contraction into FMA is disabled
 * by the build flags, so the bits do not depend on the host ISA.
 *
 * What is computed (paper references are to sections / equations / Algorithm 1):
 *   - Philox4x64-10 counter-based generator (Salmon et al., SC'11): point i uses
 *     counter (i,0,0,0) and key (seed,0).
 *   - R from (n, k, alpha) by binary search on Krioukov's approximation of the
 *     average degree (Sec. III-B "getTargetRadius", Eq. 22 of Krioukov et al.
 *     with zeta = 1).
 *   - Geometric band boundaries with ratio p (Sec. III-A).
 *   - Points: phi ~ U[0, 2pi), r by inverse CDF of Eq. 1 (Sec. II; Alg. 1).
 *   - Edge predicate: Eq. 3 (hyperbolic law of cosines) with the threshold rule
 *     dist <= R of Alg. 1, written as one fixed FP64 operation sequence.
 *   - Edge sets two ways: all pairs (the plain definition, the pairwise approach
 *     of Aldecoa et al. that Sec. II describes) and the band algorithm (Alg. 1:
 *     bands, per-band angular sort, getMinMaxPhi windows, binary search,
 *     candidate test, outward-only iteration).
 *   - Dynamic model (Sec. III-C, Algorithm 2, Theorem 1): step values from
 *     Philox counter (i,1,0,0), rotation modulo 2 pi, the radial step with
 *     reflection in the coordinate cosh(alpha r) - 1, which is uniform under
 *     Eq. 1 as Theorem 1 requires (the sinh(alpha r) of the printed algorithm
 *     is kept as an option for the test that shows it is not).
 *   - Timed CPU baseline: the band structure built once and the outward
 *     queries of a vertex set counted, OpenMP over the vertices.
 *   - Checks at scale: every edge (u, w), u < w, of a vertex range in order
 *     (windowed search of all bands), for pair-by-pair comparison of large
 *     graphs; the count of edges outside their getMinMaxPhi window (must be
 *     0); rounding diagnostics of the canonical predicate (pairs within
 *     8 u cosh r_v cosh r_w of the threshold; pairs a cancellation-free form
 *     of Eq. 3 decides otherwise, in FP64 and in long double).
 * Every function is pinned in tests/test_oracle_*.py against independent facts
 * (closed forms, mpmath, brute force, invariants, distribution tests).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define RO_OK 0
#define RO_ERR_INVALID_ARG 1
#define RO_ERR_NO_SOLUTION 2
#define RO_ERR_OOM 3
#define RO_ERR_OVERFLOW 6

#define RO_MAX_BANDS 64

/* ------------------------------------------------------------------------- */
/* Constants of the deterministic math definition (exact binary64 values).    */
/* ------------------------------------------------------------------------- */
static const double RO_PI = 0x1.921fb54442d18p+1;          /* double nearest pi   */
static const double RO_TWO_PI = 0x1.921fb54442d18p+2;      /* 2 * RO_PI (exact)   */
static const double RO_INV_LN2 = 0x1.71547652b82fep+0;     /* nearest 1/ln 2      */
static const double RO_LN2_HI = 0x1.62e42fee00000p-1;      /* ln 2, 32 bits       */
static const double RO_LN2_LO = 0x1.a39ef35793c76p-33;     /* ln 2 - LN2_HI       */
static const double RO_TWO_OVER_PI = 0x1.45f306dc9c883p-1; /* nearest 2/pi        */
static const double RO_PIO2_1 = 0x1.921fb54400000p+0;      /* pi/2, 33 bits       */
static const double RO_PIO2_2 = 0x1.0b4611a600000p-34;     /* next 33 bits        */
static const double RO_PIO2_3 = 0x1.3198a2e037073p-69;     /* rest, rounded       */
static const double RO_SQRT_HALF = 0x1.6a09e667f3bcdp-1;   /* nearest sqrt(1/2)   */

/* 1/j! as a correctly rounded quotient (j! is exact in binary64 for j <= 18)
 * and 2/(2j+1), tabulated once when the library is loaded. */
static double RO_INV_FACT[19];
static double RO_LOG_COEF[12];

__attribute__((constructor)) static void ro_init_tables(void)
{
    double f = 1.0;
    for (int j = 0; j <= 18; ++j) {
        if (j >= 2) f = f * (double)j;
        RO_INV_FACT[j] = 1.0 / f;
    }
    for (int j = 0; j <= 11; ++j) RO_LOG_COEF[j] = 2.0 / (double)(2 * j + 1);
}

static double ro_inv_fact(int j) { return RO_INV_FACT[j]; }

/* ------------------------------------------------------------------------- */
/* Philox4x64-10                                                              */
/* ------------------------------------------------------------------------- */
void ro_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counters (c0 + i, c1, c2, c3) for i in [0, count) (no carry: test helper). */
void ro_philox4x64_batch(uint64_t count, const uint64_t ctr0[4], const uint64_t key[2],
                         uint64_t *out)
{
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t c[4] = {ctr0[0] + i, ctr0[1], ctr0[2], ctr0[3]};
        ro_philox4x64(c, key, out + 4 * i);
    }
}

/* ------------------------------------------------------------------------- */
/* Deterministic FP64 elementary functions                                    */
/* ------------------------------------------------------------------------- */

/* e^x: Cody-Waite reduction x = k ln2 + t with a two-part ln 2, then the Taylor
 * polynomial of degree 13 in Horner form, then exact scaling by 2^k. */
double ro_exp(double x)
{
    if (x != x) return x;
    if (x > 708.0) return INFINITY;
    if (x < -708.0) return 0.0;
    double t = x * RO_INV_LN2;
    double kf = floor(t + 0.5);
    double hi = x - kf * RO_LN2_HI;       /* kf * LN2_HI is exact */
    double red = hi - kf * RO_LN2_LO;
    double p = ro_inv_fact(13);
    for (int j = 12; j >= 0; --j) {
        double pr = p * red;
        p = pr + ro_inv_fact(j);
    }
    return ldexp(p, (int)kf);
}

/* ln x for finite x > 0 (normal): x = m 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln m = 2 atanh(s), s = (m-1)/(m+1), atanh by its odd power series to s^23. */
double ro_log(double x)
{
    if (!(x > 0.0)) return (x == 0.0) ? -INFINITY : NAN;
    if (isinf(x)) return x;
    int e0;
    double m0 = frexp(x, &e0);            /* x = m0 * 2^e0, m0 in [0.5, 1) */
    double m;
    int e;
    if (m0 < RO_SQRT_HALF) { m = m0 * 2.0; e = e0 - 1; }
    else { m = m0; e = e0; }
    double f = m - 1.0;                    /* exact */
    double den = m + 1.0;
    double s = f / den;
    double z = s * s;
    double q = RO_LOG_COEF[11];            /* coefficients 2/(2j+1), j = 11..1 */
    for (int j = 10; j >= 1; --j) {
        double qz = q * z;
        q = qz + RO_LOG_COEF[j];
    }
    double s2 = s * 2.0;
    double sz = s * z;
    double tail = sz * q;
    double logm = s2 + tail;
    double ed = (double)e;
    double lo = ed * RO_LN2_LO;
    double mid = lo + logm;
    double hi = ed * RO_LN2_HI;            /* exact */
    return hi + mid;
}

/* cos d for d in [0, 2pi + 1): quadrant j = floor(d 2/pi + 1/2), three-part
 * pi/2 reduction, Taylor polynomials of cos (to z^8) and sin (to r z^8). */
double ro_cos(double d)
{
    double t = d * RO_TWO_OVER_PI;
    double jf = floor(t + 0.5);
    double r = d - jf * RO_PIO2_1;
    r = r - jf * RO_PIO2_2;
    r = r - jf * RO_PIO2_3;
    double z = r * r;
    /* cos r = sum_{j=0..8} (-1)^j z^j / (2j)! */
    double c = ro_inv_fact(16);
    for (int j = 7; j >= 0; --j) {
        double cz = c * z;
        double coef = ro_inv_fact(2 * j);
        if (j & 1) coef = -coef;
        c = cz + coef;
    }
    /* sin r = r * sum_{j=0..8} (-1)^j z^j / (2j+1)! */
    double s = ro_inv_fact(17);
    for (int j = 7; j >= 0; --j) {
        double sz = s * z;
        double coef = ro_inv_fact(2 * j + 1);
        if (j & 1) coef = -coef;
        s = sz + coef;
    }
    double sn = r * s;
    int q = ((int)jf) & 3;
    if (q == 0) return c;
    if (q == 1) return -sn;
    if (q == 2) return -c;
    return sn;
}

/* cosh x = (e^x + e^-x)/2 for x >= 0. */
double ro_cosh(double x)
{
    double e = ro_exp(x);
    double ie = 1.0 / e;
    double s = e + ie;
    return s * 0.5;
}

/* sinh x for x >= 0: odd Taylor series to x^15/15! below 0.5, else (e^x - e^-x)/2. */
double ro_sinh(double x)
{
    if (x < 0.5) {
        double z = x * x;
        double q = ro_inv_fact(15);
        for (int j = 13; j >= 1; j -= 2) {
            double qz = q * z;
            q = qz + ro_inv_fact(j);
        }
        return x * q;
    }
    double e = ro_exp(x);
    double ie = 1.0 / e;
    double s = e - ie;
    return s * 0.5;
}

/* ------------------------------------------------------------------------- */
/* Sec. III-B getTargetRadius: Krioukov's Eq. 22 with zeta = 1.               */
/* kbar(R) = (2/pi) xi^2 n [ e^{-R/2} + e^{-alpha R} (alpha R/2 (pi/(4 alpha^2)*/
/*            - (pi-1)/alpha + (pi-2)) - 1) ],  xi = alpha/(alpha - 1/2).     */
/* ------------------------------------------------------------------------- */
double ro_kbar(double R, uint64_t n, double alpha)
{
    double xi = alpha / (alpha - 0.5);
    double xi2 = xi * xi;
    double two_over_pi = 2.0 / RO_PI;
    double pre = two_over_pi * xi2;
    pre = pre * (double)n;
    double e1 = ro_exp(-(R * 0.5));
    double e2 = ro_exp(-(alpha * R));
    double a2 = alpha * alpha;
    double inv_a2 = 1.0 / a2;
    double pi4 = RO_PI * 0.25;
    double ta = pi4 * inv_a2;
    double tb = (RO_PI - 1.0) / alpha;
    double tc = RO_PI - 2.0;
    double inner = ta - tb;
    inner = inner + tc;
    double aR = alpha * R;
    double half_aR = aR * 0.5;
    double br = half_aR * inner;
    br = br - 1.0;
    double sec = e2 * br;
    double sum = e1 + sec;
    return pre * sum;
}

/* Binary search for R (the paper names only the method; the bracket is the
 * largest integer grid point j in [0, 255] with kbar(j) > k, and the search
 * keeps kbar(lo) > k >= kbar(hi) until lo and hi are adjacent doubles). */
int ro_target_radius(uint64_t n, double k, double alpha, double *R_out)
{
    if (n < 2 || n > 0xFFFFFFFFULL || !(alpha > 0.5) || !(alpha <= 100.0) || !(k > 0.0) ||
        !(k < 1e300))
        return RO_ERR_INVALID_ARG;
    int jstar = -1;
    for (int j = 0; j < 256; ++j)
        if (ro_kbar((double)j, n, alpha) > k) jstar = j;
    if (jstar < 0 || jstar == 255) return RO_ERR_NO_SOLUTION;
    double lo = (double)jstar, hi = (double)(jstar + 1);
    for (int it = 0; it < 200; ++it) {
        double sum = lo + hi;
        double mid = sum * 0.5;
        if (mid == lo || mid == hi) break;
        if (ro_kbar(mid, n, alpha) > k) lo = mid;
        else hi = mid;
    }
    *R_out = hi;
    return RO_OK;
}

/* Default band count: the paper uses "log n" bands; read as ceil(log2 n), >= 1. */
uint32_t ro_default_bands(uint64_t n)
{
    uint32_t B = 0;
    while (B < 63 && ((uint64_t)1 << B) < n) ++B;
    return B < 1 ? 1 : B;
}

/* Sec. III-A: c_0 = 0, widths c_{j+1} - c_j = c_1 p^j, c_1 = (1-p) R / (1 - p^B),
 * c_B = R.  p == 1 gives equal widths R/B. */
int ro_boundaries(double R, uint32_t B, double p, double *c)
{
    if (B < 1 || B > RO_MAX_BANDS || !(p > 0.0) || !(R > 0.0)) return RO_ERR_INVALID_ARG;
    c[0] = 0.0;
    if (p == 1.0) {
        for (uint32_t j = 1; j < B; ++j) c[j] = (R * (double)j) / (double)B;
    } else {
        double pw = 1.0;
        for (uint32_t j = 0; j < B; ++j) pw = pw * p;
        double num = (1.0 - p) * R;
        double c1 = num / (1.0 - pw);
        double step = c1;
        for (uint32_t j = 1; j < B; ++j) {
            double next = c[j - 1] + step;
            c[j] = next < R ? next : R;
            step = step * p;
        }
    }
    c[B] = R;
    return RO_OK;
}

/* ------------------------------------------------------------------------- */
/* Alg. 1, sampling step: phi ~ U[0,2pi), r with the density of Eq. 1.         */
/* Inverse CDF: F(r) = (cosh(alpha r) - 1)/(cosh(alpha R) - 1), so            */
/* r = acosh(1 + U (cosh(alpha R) - 1)) / alpha, acosh(1+w) = ln(1 + w +      */
/* sqrt(w (w + 2))).                                                          */
/* ------------------------------------------------------------------------- */
/* The radius of the 53-bit uniform variate ur (cm1 = cosh(alpha R) - 1). */
static double ro_radius_of(uint64_t ur, double R, double cm1, double inv_alpha)
{
    const double U53 = 0x1.0p-53;
    double U = (double)ur * U53;
    double w = U * cm1;
    double w2 = w + 2.0;
    double ww = w * w2;
    double sq = sqrt(ww);
    double y = 1.0 + w;
    y = y + sq;
    double lg = ro_log(y);
    double rr = lg * inv_alpha;
    if (rr > R) rr = R;
    return rr;
}

int ro_sample_points(uint64_t n, double alpha, double R, uint64_t seed, uint64_t first,
                     double *phi, double *r)
{
    const double S = 0x1.921fb54442d18p-51;   /* TWO_PI * 2^-53, exact */
    double aR = alpha * R;
    double cm1 = ro_cosh(aR) - 1.0;
    double inv_alpha = 1.0 / alpha;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t id = first + i;
        uint64_t ctr[4] = {id, 0, 0, 0}, key[2] = {seed, 0}, x[4];
        ro_philox4x64(ctr, key, x);
        uint64_t uphi = x[0] >> 11, ur = x[1] >> 11;
        double ph = (double)uphi * S;
        if (ph >= RO_TWO_PI) ph = nextafter(RO_TWO_PI, 0.0);
        phi[i] = ph;
        r[i] = ro_radius_of(ur, R, cm1, inv_alpha);
    }
    return RO_OK;
}

/* The sampler's radius of given 53-bit variates (the radial step of
 * ro_sample_points alone): r[i] for u[i] < 2^53. */
int ro_radius_from_u53(const uint64_t *u, uint64_t n, double alpha, double R, double *r)
{
    double cm1 = ro_cosh(alpha * R) - 1.0;
    double inv_alpha = 1.0 / alpha;
    for (uint64_t i = 0; i < n; ++i) {
        if (u[i] >> 53) return RO_ERR_INVALID_ARG;
        r[i] = ro_radius_of(u[i], R, cm1, inv_alpha);
    }
    return RO_OK;
}

/* Band of a point: the largest j in [0, B-1] with c_j <= r (Sec. III-A: slab i is
 * c_i <= r < c_{i+1}; r = c_B = R falls into the last band). */
static uint32_t ro_band_of(double rv, const double *c, uint32_t B)
{
    uint32_t b = 0;
    for (uint32_t j = 1; j < B; ++j)
        if (c[j] <= rv) b = j;
    return b;
}

/* ------------------------------------------------------------------------- */
/* The edge predicate: Eq. 3 and the rule dist <= R (Alg. 1, edge test).      */
/*   d = |phi_v - phi_w|, c = cos d, L = ch_v ch_w - (sh_v sh_w) c,           */
/*   edge iff L <= cosh R.                                                    */
/* ------------------------------------------------------------------------- */
static double ro_L(double phv, double chv, double shv, double phw, double chw, double shw)
{
    double d = fabs(phv - phw);
    double c = ro_cos(d);
    double t1 = chv * chw;
    double t2 = shv * shw;
    double t3 = t2 * c;
    return t1 - t3;
}

int ro_edge(double phv, double rv, double phw, double rw, double R)
{
    double L = ro_L(phv, ro_cosh(rv), ro_sinh(rv), phw, ro_cosh(rw), ro_sinh(rw));
    return L <= ro_cosh(R);
}

/* Canonical L for given points (test access to the exact double compared). */
double ro_edge_L(double phv, double rv, double phw, double rw)
{
    return ro_L(phv, ro_cosh(rv), ro_sinh(rv), phw, ro_cosh(rw), ro_sinh(rw));
}

typedef struct {
    uint64_t n;
    double R, coshR;
    double *ch, *sh;
} ro_pts;

static int ro_pts_init(ro_pts *P, uint64_t n, const double *r, double R)
{
    P->n = n;
    P->R = R;
    P->coshR = ro_cosh(R);
    P->ch = (double *)malloc(sizeof(double) * (n ? n : 1));
    P->sh = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (!P->ch || !P->sh) { free(P->ch); free(P->sh); return RO_ERR_OOM; }
    for (uint64_t i = 0; i < n; ++i) { P->ch[i] = ro_cosh(r[i]); P->sh[i] = ro_sinh(r[i]); }
    return RO_OK;
}

static void ro_pts_free(ro_pts *P) { free(P->ch); free(P->sh); }

/* All pairs u < v (the plain definition of the edge set).  Writes at most
 * `capacity` pairs; returns the number of edges m (or a negative status). */
int64_t ro_brute_edges(uint64_t n, const double *phi, const double *r, double R,
                       uint32_t *pairs, uint64_t capacity)
{
    ro_pts P;
    if (ro_pts_init(&P, n, r, R) != RO_OK) return -RO_ERR_OOM;
    int64_t m = 0;
    for (uint64_t u = 0; u < n; ++u)
        for (uint64_t v = u + 1; v < n; ++v) {
            double L = ro_L(phi[u], P.ch[u], P.sh[u], phi[v], P.ch[v], P.sh[v]);
            if (L <= P.coshR) {
                if ((uint64_t)m < capacity) { pairs[2 * m] = (uint32_t)u; pairs[2 * m + 1] = (uint32_t)v; }
                ++m;
            }
        }
    ro_pts_free(&P);
    return m;
}

/* All w != v with an edge to v, ascending (one row of the adjacency, O(n)). */
int64_t ro_neighbors(uint64_t v, uint64_t n, const double *phi, const double *r, double R,
                     uint32_t *out, uint64_t capacity)
{
    double coshR = ro_cosh(R);
    double chv = ro_cosh(r[v]), shv = ro_sinh(r[v]);
    int64_t m = 0;
    for (uint64_t w = 0; w < n; ++w) {
        if (w == v) continue;
        double L = ro_L(phi[v], chv, shv, phi[w], ro_cosh(r[w]), ro_sinh(r[w]));
        if (L <= coshR) {
            if ((uint64_t)m < capacity) out[m] = (uint32_t)w;
            ++m;
        }
    }
    return m;
}

/* ------------------------------------------------------------------------- */
/* Alg. 1: band data structure and the range query                            */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t B;
    double c[RO_MAX_BANDS + 1];
    uint32_t *band;       /* band of each id                          */
    uint32_t *order;      /* ids sorted by (band, phi, id)            */
    uint64_t start[RO_MAX_BANDS + 1];
    double *sphi;         /* phi in sorted order                      */
} ro_bands;

static const double *g_sort_phi;
static const uint32_t *g_sort_band;

static int ro_cmp(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    if (g_sort_band[x] != g_sort_band[y]) return g_sort_band[x] < g_sort_band[y] ? -1 : 1;
    if (g_sort_phi[x] != g_sort_phi[y]) return g_sort_phi[x] < g_sort_phi[y] ? -1 : 1;
    return x < y ? -1 : (x > y);
}

static int ro_bands_build(ro_bands *S, uint64_t n, const double *phi, const double *r,
                          double R, uint32_t B, double p)
{
    S->B = B;
    int st = ro_boundaries(R, B, p, S->c);
    if (st != RO_OK) return st;
    S->band = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    S->order = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    S->sphi = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (!S->band || !S->order || !S->sphi) return RO_ERR_OOM;
    /* Alg. 1: insert each point into the band with c_i <= r < c_{i+1}. */
    for (uint64_t i = 0; i < n; ++i) { S->band[i] = ro_band_of(r[i], S->c, B); S->order[i] = (uint32_t)i; }
    /* Alg. 1: sort the points of each band by angle (one global sort keyed by band first). */
    g_sort_phi = phi;
    g_sort_band = S->band;
    qsort(S->order, n, sizeof(uint32_t), ro_cmp);
    for (uint32_t j = 0; j <= B; ++j) S->start[j] = 0;
    for (uint64_t i = 0; i < n; ++i) S->start[S->band[i] + 1]++;
    for (uint32_t j = 0; j < B; ++j) S->start[j + 1] += S->start[j];
    for (uint64_t i = 0; i < n; ++i) S->sphi[i] = phi[S->order[i]];
    return RO_OK;
}

static void ro_bands_free(ro_bands *S) { free(S->band); free(S->order); free(S->sphi); }

/* Sec. III-B getMinMaxPhi.  For w in band i (r_w >= c_i) to be a neighbour of
 * v, cosh R >= cosh r_v cosh c_i - sinh r_v sinh c_i cos|phi_w - phi_v|, i.e.
 * the angular deviation is at most acos((cosh r_v cosh c_i - cosh R) /
 * (sinh r_v sinh c_i)).  Written in the equivalent well-conditioned form
 * sin^2(theta/2) = (b - cosh(r_v - c_i)) / (2 sinh r_v sinh c_i) and evaluated
 * with an inflated threshold b that also admits every pair the rounded FP64
 * predicate accepts: b = (cosh R + 64 u cosh r_v cosh c_{i+1}) (1 + 1e-12).
 * Returns theta (>= pi means the whole band). */
static double ro_min_max_phi(double rv, double chv, double shv, double coshR, double ci,
                             double ci1)
{
    const double u = 0x1.0p-53;
    if (ci <= 0.0 || rv <= 0.0 || shv <= 0.0) return 4.0;
    double b = coshR + 64.0 * u * chv * cosh(ci1);
    b = b * (1.0 + 1e-12);
    double num = b - cosh(rv - ci);
    double den = 2.0 * shv * sinh(ci);
    double Q = num / den;
    if (!(Q < 1.0)) return 4.0;
    if (Q < 0.0) Q = 0.0;
    double theta = 2.0 * asin(sqrt(Q));
    return theta * (1.0 + 1e-9) + 1e-12;
}

/* First index in [lo, hi) of sphi with sphi >= x. */
static uint64_t ro_lower(const double *a, uint64_t lo, uint64_t hi, double x)
{
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* First index in [lo, hi) of sphi with sphi > x. */
static uint64_t ro_upper(const double *a, uint64_t lo, uint64_t hi, double x)
{
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

typedef struct {
    int64_t candidates;   /* candidate pairs examined (each unordered pair once)    */
    int64_t near;         /* of those, |L - cosh R| <= 1e-12 cosh R                  */
    int64_t windows;      /* (v, band) windows evaluated                             */
    int64_t band8u;       /* of the candidates, |L - cosh R| <= 8 u ch_v ch_w        */
    int64_t disagree_wc;  /* decided otherwise by the well-conditioned FP64 form     */
    int64_t disagree_ld;  /* decided otherwise by the well-conditioned long double form */
} ro_stats;

#define RO_NUM_STATS 6

static void ro_stats_store(const ro_stats *s, int64_t *out)
{
    out[0] = s->candidates; out[1] = s->near; out[2] = s->windows;
    out[3] = s->band8u; out[4] = s->disagree_wc; out[5] = s->disagree_ld;
}

static void ro_stats_add(ro_stats *a, const ro_stats *b)
{
    a->candidates += b->candidates; a->near += b->near; a->windows += b->windows;
    a->band8u += b->band8u; a->disagree_wc += b->disagree_wc; a->disagree_ld += b->disagree_ld;
}

/* Diagnostics of one examined pair with canonical value L (reported, never used
 * to decide an edge).  The canonical Eq. 3 cancels: its rounding error is below
 * a few u ch_v ch_w, so only pairs within 16 u ch_v ch_w of the threshold can be
 * decided differently by a form without cancellation.  For those, Eq. 3 is
 * rewritten with cosh(a) cosh(b) - sinh(a) sinh(b) = cosh(a - b) and
 * 1 - cos d = 2 sin^2(d/2):
 *   L' = cosh(r_v - r_w) + 2 sinh r_v sinh r_w sin^2(d/2),
 * evaluated once in FP64 (libm) and once in long double (libm). */
static void ro_diagnose(double phv, double rv, double chv, double shv, double phw, double rw, double chw,
                        double shw, double L, double coshR, double R, ro_stats *st)
{
    const double u = 0x1.0p-53;
    const double dev = fabs(L - coshR);
    if (dev <= 1e-12 * coshR) st->near++;
    const double chch = chv * chw;
    if (dev <= 8.0 * u * chch) st->band8u++;
    if (dev > 16.0 * u * chch) return;
    const int edge = L <= coshR;
    double d = fabs(phv - phw);
    double sd = sin(0.5 * d);
    double Lw = cosh(rv - rw) + 2.0 * shv * shw * (sd * sd);
    if ((Lw <= cosh(R)) != edge) st->disagree_wc++;
    long double dl = fabsl((long double)phv - (long double)phw);
    long double sdl = sinl(0.5L * dl);
    long double Ll = coshl((long double)rv - (long double)rw) +
                     2.0L * sinhl((long double)rv) * sinhl((long double)rw) * (sdl * sdl);
    if ((Ll <= coshl((long double)R)) != edge) st->disagree_ld++;
}

/* The range query of Alg. 1 for the vertices v in [v0, v1) (ids).  For each
 * band i with c_{i+1} > r_v -- read as every band from v's own band outward --
 * candidates w come from the getMinMaxPhi window found by binary search in the
 * band's angle-sorted list.  Cross-band edges are found from the inner end only;
 * a same-band edge is reported from its endpoint with the smaller id. */
static int64_t ro_query_range(const ro_bands *S, const ro_pts *P, const double *phi,
                              const double *r, uint64_t v0, uint64_t v1, uint32_t *pairs,
                              uint64_t capacity, int64_t m0, ro_stats *st)
{
    int64_t m = m0;
    for (uint64_t v = v0; v < v1; ++v) {
        uint32_t bv = S->band[v];
        for (uint32_t i = bv; i < S->B; ++i) {
            uint64_t s = S->start[i], e = S->start[i + 1];
            if (s == e) continue;
            st->windows++;
            double th = ro_min_max_phi(r[v], P->ch[v], P->sh[v], P->coshR, S->c[i], S->c[i + 1]);
            uint64_t ranges[2][2];
            int nr = 0;
            if (th >= RO_PI) {
                ranges[0][0] = s; ranges[0][1] = e; nr = 1;
            } else {
                double lo = phi[v] - th, hi = phi[v] + th;
                if (lo < 0.0) {
                    ranges[0][0] = ro_lower(S->sphi, s, e, lo + RO_TWO_PI); ranges[0][1] = e;
                    ranges[1][0] = s; ranges[1][1] = ro_upper(S->sphi, s, e, hi);
                    nr = 2;
                } else if (hi >= RO_TWO_PI) {
                    ranges[0][0] = ro_lower(S->sphi, s, e, lo); ranges[0][1] = e;
                    ranges[1][0] = s; ranges[1][1] = ro_upper(S->sphi, s, e, hi - RO_TWO_PI);
                    nr = 2;
                } else {
                    ranges[0][0] = ro_lower(S->sphi, s, e, lo);
                    ranges[0][1] = ro_upper(S->sphi, s, e, hi);
                    nr = 1;
                }
                /* the two pieces of a wrapped window overlap only if they cover the band */
                if (nr == 2 && ranges[1][1] > ranges[0][0]) {
                    ranges[0][0] = s; ranges[0][1] = e; nr = 1;
                }
            }
            for (int k = 0; k < nr; ++k)
                for (uint64_t q = ranges[k][0]; q < ranges[k][1]; ++q) {
                    uint32_t w = S->order[q];
                    if (w == v) continue;
                    if (i == bv && w < v) continue;
                    st->candidates++;
                    double L = ro_L(phi[v], P->ch[v], P->sh[v], phi[w], P->ch[w], P->sh[w]);
                    ro_diagnose(phi[v], r[v], P->ch[v], P->sh[v], phi[w], r[w], P->ch[w], P->sh[w], L, P->coshR,
                                P->R, st);
                    if (L <= P->coshR) {
                        if ((uint64_t)m < capacity) {
                            pairs[2 * m] = (uint32_t)(v < w ? v : w);
                            pairs[2 * m + 1] = (uint32_t)(v < w ? w : v);
                        }
                        ++m;
                    }
                }
        }
    }
    return m;
}

/* Full band algorithm (Alg. 1) on given points; stats[6] = {candidates, near,
 * windows, band8u, disagree_wc, disagree_ld} (see ro_stats). */
int64_t ro_band_edges(uint64_t n, const double *phi, const double *r, double R, uint32_t B,
                      double p, uint32_t *pairs, uint64_t capacity, int64_t *stats)
{
    ro_pts P;
    ro_bands S;
    memset(&S, 0, sizeof(S));
    if (ro_pts_init(&P, n, r, R) != RO_OK) return -RO_ERR_OOM;
    int st = ro_bands_build(&S, n, phi, r, R, B, p);
    if (st != RO_OK) { ro_pts_free(&P); ro_bands_free(&S); return -st; }
    ro_stats s;
    memset(&s, 0, sizeof(s));
    int64_t m = ro_query_range(&S, &P, phi, r, 0, n, pairs, capacity, 0, &s);
    if (stats) ro_stats_store(&s, stats);
    ro_pts_free(&P);
    ro_bands_free(&S);
    return m;
}

/* Band structure accessors for tests: band of each id and the boundaries. */
int ro_band_assign(uint64_t n, const double *r, double R, uint32_t B, double p, uint32_t *band)
{
    double c[RO_MAX_BANDS + 1];
    int st = ro_boundaries(R, B, p, c);
    if (st != RO_OK) return st;
    for (uint64_t i = 0; i < n; ++i) band[i] = ro_band_of(r[i], c, B);
    return RO_OK;
}

/* Timed CPU baseline: the band algorithm over the given vertex ids, counting
 * edges (no output), OpenMP-parallel over the ids when built with OpenMP.
 * Returns the edge count; *threads receives the number of threads used and
 * stats (if not NULL) the RO_NUM_STATS counters of ro_stats. */
static int64_t ro_count_ids(const ro_bands *S, const ro_pts *P, const double *phi, const double *r,
                            const uint32_t *ids, uint64_t nids, int32_t *threads, int64_t *stats)
{
    int64_t m = 0;
    int nt = 1;
    ro_stats tot;
    memset(&tot, 0, sizeof(tot));
#ifdef _OPENMP
#pragma omp parallel reduction(+ : m)
    {
        ro_stats loc;
        memset(&loc, 0, sizeof(loc));
#pragma omp single
        nt = omp_get_num_threads();
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < (int64_t)nids; ++q)
            m += ro_query_range(S, P, phi, r, ids[q], (uint64_t)ids[q] + 1, NULL, 0, 0, &loc);
#pragma omp critical
        ro_stats_add(&tot, &loc);
    }
#else
    for (uint64_t q = 0; q < nids; ++q)
        m += ro_query_range(S, P, phi, r, ids[q], (uint64_t)ids[q] + 1, NULL, 0, 0, &tot);
#endif
    if (threads) *threads = nt;
    if (stats) ro_stats_store(&tot, stats);
    return m;
}

int64_t ro_band_count_subset(uint64_t n, const double *phi, const double *r, double R,
                             uint32_t B, double p, const uint32_t *ids, uint64_t nids,
                             int32_t *threads, int64_t *stats)
{
    ro_pts P;
    ro_bands S;
    memset(&S, 0, sizeof(S));
    if (ro_pts_init(&P, n, r, R) != RO_OK) return -RO_ERR_OOM;
    int st = ro_bands_build(&S, n, phi, r, R, B, p);
    if (st != RO_OK) { ro_pts_free(&P); ro_bands_free(&S); return -st; }
    int64_t m = ro_count_ids(&S, &P, phi, r, ids, nids, threads, stats);
    ro_pts_free(&P);
    ro_bands_free(&S);
    return m;
}

/* Threads of the calling thread's next OpenMP regions (the timed baseline is
 * reported on one thread and on all cores); nt <= 0 restores the default. */
void ro_set_threads(int32_t nt)
{
#ifdef _OPENMP
    static int initial = 0;
    if (!initial) initial = omp_get_max_threads();
    omp_set_num_threads(nt > 0 ? nt : initial);
#else
    (void)nt;
#endif
}

int ro_openmp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The constants above, in order, for tests that check them against their
 * mathematical definitions: PI, TWO_PI, INV_LN2, LN2_HI, LN2_LO, TWO_OVER_PI,
 * PIO2_1, PIO2_2, PIO2_3, SQRT_HALF. */
void ro_constants(double *out)
{
    out[0] = RO_PI; out[1] = RO_TWO_PI; out[2] = RO_INV_LN2; out[3] = RO_LN2_HI;
    out[4] = RO_LN2_LO; out[5] = RO_TWO_OVER_PI; out[6] = RO_PIO2_1; out[7] = RO_PIO2_2;
    out[8] = RO_PIO2_3; out[9] = RO_SQRT_HALF;
}

/* The same band structure built once and queried many times (timed CPU baseline). */
typedef struct {
    uint64_t n;
    const double *phi, *r;
    ro_pts P;
    ro_bands S;
} ro_prepared;

void *ro_prepare(uint64_t n, const double *phi, const double *r, double R, uint32_t B, double p)
{
    ro_prepared *h = (ro_prepared *)calloc(1, sizeof(ro_prepared));
    if (!h) return NULL;
    h->n = n;
    h->phi = phi;
    h->r = r;
    if (ro_pts_init(&h->P, n, r, R) != RO_OK) { free(h); return NULL; }
    if (ro_bands_build(&h->S, n, phi, r, R, B, p) != RO_OK) {
        ro_pts_free(&h->P);
        ro_bands_free(&h->S);
        free(h);
        return NULL;
    }
    return h;
}

int64_t ro_prepared_count(void *handle, const uint32_t *ids, uint64_t nids, int32_t *threads, int64_t *stats)
{
    ro_prepared *h = (ro_prepared *)handle;
    return ro_count_ids(&h->S, &h->P, h->phi, h->r, ids, nids, threads, stats);
}

void ro_prepared_free(void *handle)
{
    ro_prepared *h = (ro_prepared *)handle;
    if (!h) return;
    ro_pts_free(&h->P);
    ro_bands_free(&h->S);
    free(h);
}

/* Is phw inside the angular window [phv - th, phv + th] (modulo 2 pi)?  The same
 * membership the range query's binary searches give (both ends included). */
static int ro_in_window(double phv, double th, double phw)
{
    if (th >= RO_PI) return 1;
    double lo = phv - th, hi = phv + th;
    if (lo < 0.0) return phw >= lo + RO_TWO_PI || phw <= hi;
    if (hi >= RO_TWO_PI) return phw >= lo || phw <= hi - RO_TWO_PI;
    return lo <= phw && phw <= hi;
}

static int ro_cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y);
}

/* Neighbours w > u of one vertex u, ascending, appended to *buf (grown as needed).
 * Every band is searched (inward as well as outward): getMinMaxPhi's window at a
 * band's inner radius bounds the angle of every neighbour in that band, whichever
 * side of u the band lies (Sec. III-B: for b >= cosh r_u the admissible angle
 * grows with r_w, so the inner radius is the worst case).  Returns the new length
 * or -1 when out of memory. */
static int64_t ro_upper_neighbors_one(const ro_bands *S, const ro_pts *P, const double *phi, const double *r,
                                      uint64_t u, uint32_t **buf, uint64_t *cap, uint64_t len)
{
    uint64_t first = len;
    for (uint32_t i = 0; i < S->B; ++i) {
        uint64_t s = S->start[i], e = S->start[i + 1];
        if (s == e) continue;
        double th = ro_min_max_phi(r[u], P->ch[u], P->sh[u], P->coshR, S->c[i], S->c[i + 1]);
        uint64_t ranges[2][2];
        int nr;
        if (th >= RO_PI) {
            ranges[0][0] = s; ranges[0][1] = e; nr = 1;
        } else {
            double lo = phi[u] - th, hi = phi[u] + th;
            if (lo < 0.0) {
                ranges[0][0] = ro_lower(S->sphi, s, e, lo + RO_TWO_PI); ranges[0][1] = e;
                ranges[1][0] = s; ranges[1][1] = ro_upper(S->sphi, s, e, hi);
                nr = 2;
            } else if (hi >= RO_TWO_PI) {
                ranges[0][0] = ro_lower(S->sphi, s, e, lo); ranges[0][1] = e;
                ranges[1][0] = s; ranges[1][1] = ro_upper(S->sphi, s, e, hi - RO_TWO_PI);
                nr = 2;
            } else {
                ranges[0][0] = ro_lower(S->sphi, s, e, lo);
                ranges[0][1] = ro_upper(S->sphi, s, e, hi);
                nr = 1;
            }
            if (nr == 2 && ranges[1][1] > ranges[0][0]) {
                ranges[0][0] = s; ranges[0][1] = e; nr = 1;
            }
        }
        for (int k = 0; k < nr; ++k)
            for (uint64_t q = ranges[k][0]; q < ranges[k][1]; ++q) {
                uint32_t w = S->order[q];
                if (w <= u) continue;
                double L = ro_L(phi[u], P->ch[u], P->sh[u], phi[w], P->ch[w], P->sh[w]);
                if (L > P->coshR) continue;
                if (len == *cap) {
                    uint64_t nc = *cap ? 2 * *cap : 4096;
                    uint32_t *nb = (uint32_t *)realloc(*buf, sizeof(uint32_t) * 2 * nc);
                    if (!nb) return -1;
                    *buf = nb;
                    *cap = nc;
                }
                (*buf)[2 * len] = (uint32_t)u;
                (*buf)[2 * len + 1] = w;
                ++len;
            }
    }
    /* one vertex's pairs share u: sorting the (u, w) records by w sorts the row */
    uint64_t cnt = len - first;
    if (cnt > 1) {
        uint32_t *row = (uint32_t *)malloc(sizeof(uint32_t) * cnt);
        if (!row) return -1;
        for (uint64_t j = 0; j < cnt; ++j) row[j] = (*buf)[2 * (first + j) + 1];
        qsort(row, cnt, sizeof(uint32_t), ro_cmp_u32);
        for (uint64_t j = 0; j < cnt; ++j) (*buf)[2 * (first + j) + 1] = row[j];
        free(row);
    }
    return (int64_t)len;
}

/* Every edge (u, w) with u in [u0, u1) and u < w, in lexicographic order: the
 * edge set of the plain definition cut into vertex ranges, so that a large graph
 * can be compared pair by pair one range at a time.  OpenMP over u with a static
 * schedule (thread t owns the t-th contiguous block of u, so concatenating the
 * threads' buffers in thread order keeps the order).  Writes the pairs when they
 * fit into `capacity`; returns m (or a negative status). */
int64_t ro_prepared_upper_pairs(void *handle, uint64_t u0, uint64_t u1, uint32_t *pairs, uint64_t capacity)
{
    ro_prepared *h = (ro_prepared *)handle;
    if (!h || u1 > h->n || u0 > u1) return -RO_ERR_INVALID_ARG;
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    uint32_t **bufs = (uint32_t **)calloc((size_t)nt, sizeof(uint32_t *));
    uint64_t *lens = (uint64_t *)calloc((size_t)nt, sizeof(uint64_t));
    int failed = 0;
    if (!bufs || !lens) { free(bufs); free(lens); return -RO_ERR_OOM; }
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        uint64_t cap = 0, len = 0;
        uint32_t *buf = NULL;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t u = (int64_t)u0; u < (int64_t)u1; ++u) {
            int f;
#ifdef _OPENMP
#pragma omp atomic read
#endif
            f = failed;
            if (f) continue;
            int64_t nl = ro_upper_neighbors_one(&h->S, &h->P, h->phi, h->r, (uint64_t)u, &buf, &cap, len);
            if (nl < 0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                failed = 1;
            } else {
                len = (uint64_t)nl;
            }
        }
        bufs[t] = buf;
        lens[t] = len;
    }
    uint64_t m = 0;
    for (int t = 0; t < nt; ++t) m += lens[t];
    if (!failed && m <= capacity) {
        uint64_t at = 0;
        for (int t = 0; t < nt; ++t) {
            if (lens[t]) memcpy(pairs + 2 * at, bufs[t], sizeof(uint32_t) * 2 * lens[t]);
            at += lens[t];
        }
    }
    for (int t = 0; t < nt; ++t) free(bufs[t]);
    free(bufs);
    free(lens);
    return failed ? -RO_ERR_OOM : (int64_t)m;
}

/* Window check at scale (Sec. III-B getMinMaxPhi): for each listed vertex v, every
 * edge (v, w) of the plain definition (all n points tested) must lie inside v's
 * window for w's band, evaluated at that band's inner radius, inward bands
 * included.  out[0] = edges examined, out[1] = edges outside their window (must be
 * 0), out[2] = edges found by Alg. 1 from v's side (outward bands, same band from
 * the smaller id), out[3] = edges of v whose inner endpoint is v by that rule.
 * theta_scale multiplies every window narrower than the whole band: 1 for the
 * check, below 1 for the test that shows the check detects narrow windows.
 * OpenMP over the listed vertices. */
int ro_prepared_window_misses(void *handle, const uint32_t *ids, uint64_t nids, double theta_scale, int64_t *out)
{
    ro_prepared *h = (ro_prepared *)handle;
    if (!h || !out) return RO_ERR_INVALID_ARG;
    int64_t edges = 0, misses = 0, alg1 = 0, owned = 0;
    const ro_bands *S = &h->S;
    const ro_pts *P = &h->P;
    const double *phi = h->phi, *r = h->r;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : edges, misses, alg1, owned)
#endif
    for (int64_t q = 0; q < (int64_t)nids; ++q) {
        uint64_t v = ids[q];
        if (v >= h->n) continue;
        double th[RO_MAX_BANDS];
        for (uint32_t i = 0; i < S->B; ++i) {
            th[i] = ro_min_max_phi(r[v], P->ch[v], P->sh[v], P->coshR, S->c[i], S->c[i + 1]);
            if (th[i] < RO_PI) th[i] = th[i] * theta_scale;
        }
        uint32_t bv = S->band[v];
        for (uint64_t w = 0; w < h->n; ++w) {
            if (w == v) continue;
            double L = ro_L(phi[v], P->ch[v], P->sh[v], phi[w], P->ch[w], P->sh[w]);
            if (L > P->coshR) continue;
            ++edges;
            uint32_t bw = S->band[w];
            if (!ro_in_window(phi[v], th[bw], phi[w])) ++misses;
            if (bw > bv || (bw == bv && w > v)) ++owned;
        }
        ro_stats st;
        memset(&st, 0, sizeof(st));
        alg1 += ro_query_range(S, P, phi, r, v, v + 1, NULL, 0, 0, &st);
    }
    out[0] = edges;
    out[1] = misses;
    out[2] = alg1;
    out[3] = owned;
    return RO_OK;
}

/* ------------------------------------------------------------------------- */
/* Dynamic model (Sec. III-C; Algorithm 2, radial movement; Theorem 1).       */
/*                                                                            */
/* Step values of node i: Philox counter (i, 1, 0, 0), key (seed, 0), words    */
/* x0, x1; U = (x >> 11) * 2^-53; tau_phi = lo_phi + (hi_phi - lo_phi) * U0,   */
/* tau_r = lo_r + (hi_r - lo_r) * U1.                                         */
/*                                                                            */
/* One movement step of node i, in place:                                     */
/*   rotation   p = phi + tau_phi, brought into [0, 2pi) by subtracting or     */
/*              adding 2pi (a sum that rounds up to 2pi becomes the largest    */
/*              double below 2pi);                                            */
/*   radial     the radius is mapped to a coordinate x, moved to y = x + tau_r */
/*              and mapped back; while y is outside [0, top] the step is       */
/*              mirrored at the boundary it crossed (y = 2 top - y, or y = -y) */
/*              and tau_r changes sign (the node bounces).                    */
/* Theorem 1 needs x to be uniformly distributed when r follows Eq. 1 (the      */
/* figure of Sec. III-C says so of its coordinate): then a reflected walk of   */
/* x keeps the density.  Under Eq. 1 the CDF is (cosh(alpha r) - 1) /           */
/* (cosh(alpha R) - 1), so the uniform coordinate is                           */
/*   coord 0:   x = cosh(alpha r) - 1 = 2 sinh^2(alpha r / 2), top = cosh(alpha R) - 1, */
/*              r = 2 asinh(sqrt(y / 2)) / alpha;                              */
/* Algorithm 2 as printed maps to sinh(alpha r), whose density under Eq. 1 is  */
/* x / ((cosh(alpha R) - 1) sqrt(1 + x^2)), not uniform (the proof omits the    */
/* Jacobian of the map); it is kept as                                         */
/*   coord 1:   x = sinh(alpha r), top = sinh(alpha R), r = asinh(y) / alpha,  */
/* and the tests show that it does not keep Eq. 1 while coord 0 does.         */
/*   asinh(y) = log(y + sqrt(y*y + 1)) for y >= 0, each operation rounded.     */
/* The way back is capped at R.                                               */
/* ------------------------------------------------------------------------- */
double ro_asinh(double y)
{
    double yy = y * y;
    double t = yy + 1.0;
    double s = sqrt(t);
    double u = y + s;
    return ro_log(u);
}

void ro_draw_movement(uint64_t n, uint64_t seed, double phi_lo, double phi_hi, double r_lo, double r_hi,
                      double *tau_phi, double *tau_r)
{
    const double U53 = 0x1.0p-53;
    double wphi = phi_hi - phi_lo, wr = r_hi - r_lo;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t ctr[4] = {i, 1, 0, 0}, key[2] = {seed, 0}, x[4];
        ro_philox4x64(ctr, key, x);
        double u0 = (double)(x[0] >> 11) * U53;
        double u1 = (double)(x[1] >> 11) * U53;
        double a = wphi * u0;
        double b = wr * u1;
        tau_phi[i] = phi_lo + a;
        tau_r[i] = r_lo + b;
    }
}

void ro_move(uint64_t count, const uint32_t *ids, double *phi, double *r, const double *tau_phi, double *tau_r,
             double R, double alpha, int32_t coord)
{
    double aR = alpha * R;
    const double top = coord == 1 ? ro_sinh(aR) : ro_cosh(aR) - 1.0;
    const double inv_alpha = 1.0 / alpha;
    const double below = nextafter(RO_TWO_PI, 0.0);
    for (uint64_t j = 0; j < count; ++j) {
        uint32_t i = ids[j];
        double p = phi[i] + tau_phi[i];
        for (int it = 0; it < 64 && p >= RO_TWO_PI; ++it) p = p - RO_TWO_PI;
        for (int it = 0; it < 64 && p < 0.0; ++it) p = p + RO_TWO_PI;
        if (p >= RO_TWO_PI) p = below;
        if (p < 0.0) p = 0.0;
        double tr = tau_r[i];
        double ar = alpha * r[i];
        double x;
        if (coord == 1) {
            x = ro_sinh(ar);
        } else {
            double half = ar * 0.5;
            double sh = ro_sinh(half);
            double sq = sh * sh;
            x = sq * 2.0;
        }
        double y = x + tr;
        for (int it = 0; it < 64 && (y > top || y < 0.0); ++it) {
            if (y > top) {
                double t2 = top + top;
                y = t2 - y;
            } else {
                y = -y;
            }
            tr = -tr;
        }
        if (y > top) y = top;
        if (y < 0.0) y = 0.0;
        double z;
        if (coord == 1) {
            z = ro_asinh(y) * inv_alpha;
        } else {
            double hy = y * 0.5;
            double sy = sqrt(hy);
            double as = ro_asinh(sy);
            double two = as * 2.0;
            z = two * inv_alpha;
        }
        if (z > R) z = R;
        phi[i] = p;
        r[i] = z;
        tau_r[i] = tr;
    }
}
