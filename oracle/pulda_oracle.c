/*
 * pulda_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * Polya-urn partially collapsed LDA sampler (Terenin, Magnusson, Jonsson,
 * Draper, arXiv 1704.03581).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may build, load or call it.  It shares no code,
 * header, table or constant generator with the CUDA library: every table and
 * every draw below is computed here, from the paper and from the published
 * definitions of the building blocks (Philox4x32-10, Walker/Vose alias method).
 *
 * Everything is dense and written loop by loop so it can be read against the
 * paper:
 *   - counts n_{k,v}, m_{d,k}: notation table, Section 1;
 *   - Phi-step: Definition "Poisson Polya Urn" (Section 3.3), Eq. (7)
 *     (rates beta + n_{k,v}), Algorithm 2 first bullet, and "Efficient
 *     sampling of Phi" (alias tables for rate beta+l, l <= L = 100; rounded
 *     Gaussian above L);
 *   - z-step: Algorithm 2 second bullet and "Efficient sampling of z"
 *     (a/b split, sigma_a + sigma_b, alias table for the a part, iterate the
 *     b part).
 *
 * Where the paper is silent the oracle follows these readings (they are the
 * same readings the CUDA path follows, restated independently there):
 *   R-RNG  counter-based Philox4x32-10 keyed by the 64-bit seed; counter =
 *          (c0, c1, sweep, tag<<28 | aux).
 *   R-POIS Pois(beta+l), l in 1..L, by an integer Walker/Vose alias table whose
 *          support is every j with pmf(j) >= 2^-40 * pmf(mode); weights
 *          floor(2^40 * pmf(j)/pmf(mode) + 1/2).
 *   R-BETA entries with n_{k,v} = 0 draw Pois(beta) by skipping ahead: gaps
 *          between nonzero draws are Geometric(1 - e^-beta) (inverted from a
 *          uint32 CDF table), the value at a hit is zero-truncated Pois(beta).
 *   R-GAUSS l > L: c = max(0, floor(mu + sqrt(mu) g + 1/2)), mu = beta + l,
 *          g from a 2^16-cell equiprobable inverse-normal table, linear in the
 *          cell.
 *   R-DEAD a row with S_k = 0 is redrawn whole, attempt a = 1, 2, ..., until
 *          S_k > 0 (zero-truncation of the hierarchical representation, Eq. 8).
 *   R-FIX  the z conditional is evaluated in exact integer arithmetic:
 *          phi is quantised per word to 24 bits relative to the column max
 *          (q >= 1 for every nonzero), alpha terms to 2^-16 units; all sums
 *          are exact 64-bit integers, so summation order cannot change a draw.
 *   R-ZERO a token whose conditional has zero total mass keeps its topic.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 *        pulda_oracle.c -lm
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "pulda_oracle.h"

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As    */
/* Easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, with a  */
/* Weyl key schedule.                                                         */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t sweep,
                  uint32_t tag, uint32_t aux, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, sweep, (tag << 28) | (aux & 0x0FFFFFFFu)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox(ctr, key, out);
}

/* Index in [0, n) from a 32-bit word: floor(x * n / 2^32). */
static uint32_t scale32(uint32_t x, uint32_t n)
{
    return (uint32_t)(((uint64_t)x * n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Walker alias tables, built with Vose's method in exact integer arithmetic */
/* (Walker 1977, cited in "Efficient sampling of Phi"; Vose 1991).           */
/* Slot s is kept when a uniform 32-bit word is < thr[s], else alias[s].     */
/* ------------------------------------------------------------------------ */
uint64_t or_vose(const uint64_t *W, int32_t n, uint32_t *thr, int32_t *alias)
{
    uint64_t T = 0;
    for (int32_t j = 0; j < n; j++) T += W[j];
    if (T == 0) {
        for (int32_t j = 0; j < n; j++) { thr[j] = 0xFFFFFFFFu; alias[j] = j; }
        return 0;
    }
    uint64_t *P = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int32_t *small = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *large = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t ns = 0, nl = 0;
    /* Scale so that every slot holds exactly T units of mass. */
    for (int32_t j = 0; j < n; j++) P[j] = W[j] * (uint64_t)n;
    for (int32_t j = 0; j < n; j++) {
        if (P[j] < T) small[ns++] = j; else large[nl++] = j;
    }
    while (ns > 0 && nl > 0) {
        int32_t s = small[--ns];
        int32_t l = large[--nl];
        thr[s] = (uint32_t)(((unsigned __int128)P[s] << 32) / T);
        alias[s] = l;
        P[l] = P[l] - (T - P[s]);           /* l donates what s is missing */
        if (P[l] < T) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int32_t l = large[--nl]; thr[l] = 0xFFFFFFFFu; alias[l] = l; }
    while (ns > 0) { int32_t s = small[--ns]; thr[s] = 0xFFFFFFFFu; alias[s] = s; }
    free(P); free(small); free(large);
    return T;
}

/* ------------------------------------------------------------------------ */
/* Poisson pmf weights relative to the mode, truncated where the pmf drops   */
/* below 2^-40 of the mode's.  jmin = 1 gives the zero-truncated law.        */
/* pmf(j+1)/pmf(j) = lam/(j+1): no exponential is needed for ratios.         */
/* ------------------------------------------------------------------------ */
#define TRUNC_REL 9.094947017729282e-13 /* 2^-40 */

int32_t or_pois_weights(double lam, int32_t jmin, int32_t cap,
                        int64_t *lo_out, uint64_t *W)
{
    int64_t mode = (int64_t)floor(lam);
    if (mode < jmin) mode = jmin;
    double *down = (double *)malloc(sizeof(double) * (size_t)cap);
    double *wt = (double *)malloc(sizeof(double) * (size_t)cap);
    int32_t nb = 0, n = 0;
    double w = 1.0;
    /* below the mode: pmf(j-1) = pmf(j) * j / lam */
    for (int64_t j = mode; j > jmin; j--) {
        double wn = w * (double)j / lam;
        if (wn < TRUNC_REL) break;
        if (nb + 2 > cap) { free(down); free(wt); return -1; }
        down[nb++] = wn;
        w = wn;
    }
    for (int32_t t = nb - 1; t >= 0; t--) wt[n++] = down[t];
    wt[n++] = 1.0;                           /* the mode itself */
    /* above the mode: pmf(j+1) = pmf(j) * lam / (j+1) */
    w = 1.0;
    for (int64_t j = mode;; j++) {
        double wn = w * lam / (double)(j + 1);
        if (wn < TRUNC_REL) break;
        if (n + 1 > cap) { free(down); free(wt); return -1; }
        wt[n++] = wn;
        w = wn;
    }
    for (int32_t j = 0; j < n; j++) W[j] = (uint64_t)floor(wt[j] * 1099511627776.0 + 0.5); /* 2^40 */
    *lo_out = mode - nb;
    free(down); free(wt);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Tables for one beta.                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t lo;
    int32_t n;
    uint32_t *thr;
    int32_t *alias;
} or_table;

struct or_ctx {
    double beta;
    or_table pois[OR_L + 1];      /* index l = 1..L : Pois(beta + l) */
    or_table ztp;                 /* zero-truncated Pois(beta) */
    uint32_t geo[OR_LG];          /* P(gap <= g) * 2^32, g = 0..LG-1 */
    double gauss_q[OR_GAUSS_CELLS + 1];
};

static int build_table(double lam, int32_t jmin, or_table *t)
{
    int32_t cap = 4096;
    uint64_t *W = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)cap);
    int32_t n = or_pois_weights(lam, jmin, cap, &t->lo, W);
    if (n <= 0) { free(W); return -1; }
    t->n = n;
    t->thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    t->alias = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    or_vose(W, n, t->thr, t->alias);
    free(W);
    return 0;
}

/* Standard normal CDF through libm's erfc. */
static double norm_cdf(double x) { return 0.5 * erfc(-x * 0.70710678118654752440); }

/* Inverse normal CDF by bisection: the smallest representable x the
   bisection reaches with norm_cdf(x) >= p. */
double or_norm_quantile(double p)
{
    double lo = -40.0, hi = 40.0;
    for (int it = 0; it < 2000; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (norm_cdf(mid) < p) lo = mid; else hi = mid;
    }
    return hi;
}

/* Q[i] = Phi^{-1}(i / 2^16) for 0 < i < 2^16, the two outer edges at
   Phi^{-1}(2^-24) and its mirror.  The lower half is found by bisection (where
   the normal CDF is resolved finely); the upper half is its mirror image, as
   the normal law is symmetric, and Q[2^15] = 0. */
void or_gauss_table(double *Q)
{
    const double cells = (double)OR_GAUSS_CELLS;
    const int half = OR_GAUSS_CELLS / 2;
    Q[0] = or_norm_quantile(OR_GAUSS_TAIL_P);
    for (int i = 1; i < half; i++) Q[i] = or_norm_quantile((double)i / cells);
    Q[half] = 0.0;
    for (int i = 0; i < half; i++) Q[OR_GAUSS_CELLS - i] = -Q[i];
}

void or_geo_table(double beta, uint32_t *thr)
{
    for (int g = 0; g < OR_LG; g++) {
        /* P(G <= g) = 1 - e^{-beta (g+1)} for G ~ Geometric(1 - e^{-beta}) */
        double cdf = -expm1(-beta * (double)(g + 1));
        double t = floor(cdf * 4294967296.0);
        thr[g] = t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
    }
}

or_ctx *or_ctx_new(float beta_f)
{
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->beta = (double)beta_f;
    for (int l = 1; l <= OR_L; l++)
        if (build_table(c->beta + (double)l, 0, &c->pois[l]) != 0) { or_ctx_free(c); return NULL; }
    if (build_table(c->beta, 1, &c->ztp) != 0) { or_ctx_free(c); return NULL; }
    or_geo_table(c->beta, c->geo);
    or_gauss_table(c->gauss_q);
    return c;
}

void or_ctx_free(or_ctx *c)
{
    if (!c) return;
    for (int l = 0; l <= OR_L; l++) { free(c->pois[l].thr); free(c->pois[l].alias); }
    free(c->ztp.thr); free(c->ztp.alias);
    free(c);
}

int32_t or_ctx_table(const or_ctx *c, int32_t which, int64_t *lo, uint32_t *thr, int32_t *alias)
{
    const or_table *t = which == 0 ? &c->ztp : &c->pois[which];
    if (which < 0 || which > OR_L) return -1;
    if (thr) memcpy(thr, t->thr, sizeof(uint32_t) * (size_t)t->n);
    if (alias) memcpy(alias, t->alias, sizeof(int32_t) * (size_t)t->n);
    if (lo) *lo = t->lo;
    return t->n;
}

void or_ctx_geo(const or_ctx *c, uint32_t *thr) { memcpy(thr, c->geo, sizeof(c->geo)); }
void or_ctx_gauss(const or_ctx *c, double *Q) { memcpy(Q, c->gauss_q, sizeof(c->gauss_q)); }

static int64_t alias_draw(const or_table *t, uint32_t xs, uint32_t xa)
{
    uint32_t s = scale32(xs, (uint32_t)t->n);
    int32_t j = xa < t->thr[s] ? (int32_t)s : t->alias[s];
    return t->lo + j;
}

/* Gaussian draw g from the inverse-CDF table: cell from the top 16 bits of
   x0, position inside the cell from the remaining 48 bits of (x0, x1). */
double or_gauss_draw(const or_ctx *c, uint32_t x0, uint32_t x1)
{
    uint32_t cell = x0 >> 16;
    uint64_t frac48 = ((uint64_t)(x0 & 0xFFFFu) << 32) | x1;
    double f = (double)frac48 * 3.552713678800501e-15; /* 2^-48 */
    double a = c->gauss_q[cell], b = c->gauss_q[cell + 1];
    return a + (b - a) * f;
}

/* One entry of Phi's count matrix: c ~ Pois(beta + l), l >= 1. */
uint32_t or_draw_entry(const or_ctx *c, int64_t l, uint32_t x0, uint32_t x1)
{
    if (l <= OR_L) return (uint32_t)alias_draw(&c->pois[l], x0, x1);
    double mu = c->beta + (double)l;
    double sd = sqrt(mu);
    double g = or_gauss_draw(c, x0, x1);
    double y = mu + sd * g;
    double r = floor(y + 0.5);
    if (r < 0.0) r = 0.0;
    if (r > 4294967295.0) r = 4294967295.0;
    return (uint32_t)r;
}

/* Smallest g in [0, LG) with x < geo[g]; -1 when the gap is >= LG. */
static int32_t geo_gap(const or_ctx *c, uint32_t x)
{
    for (int32_t g = 0; g < OR_LG; g++)
        if (x < c->geo[g]) return g;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Initial topics (the paper does not say how to start the chain): uniform. */
/* ------------------------------------------------------------------------ */
void or_init_z(int64_t N, int32_t K, uint64_t seed, int64_t index_base, int16_t *z)
{
    for (int64_t i = 0; i < N; i++) {
        uint64_t t = (uint64_t)(index_base + i);
        uint32_t x[4];
        draw4(seed, (uint32_t)t, (uint32_t)(t >> 32), 0, OR_TAG_INIT, 0, x);
        z[i] = (int16_t)scale32(x[0], (uint32_t)K);
    }
}

/* n_{k,v}: number of tokens of word type v assigned to topic k (notation
   table).  Stored word-major: n_vk[v*K + k]. */
void or_count_n(int64_t N, const int32_t *w, const int16_t *z, int32_t K, int32_t V, int32_t *n_vk)
{
    memset(n_vk, 0, sizeof(int32_t) * (size_t)K * (size_t)V);
    for (int64_t i = 0; i < N; i++) n_vk[(int64_t)w[i] * K + z[i]] += 1;
}

/* m_{d,k}: number of tokens of document d assigned to topic k. */
void or_doc_topic(const int64_t *doc_off, int64_t D, const int16_t *z, int32_t K, int32_t *m_dk)
{
    memset(m_dk, 0, sizeof(int32_t) * (size_t)D * (size_t)K);
    for (int64_t d = 0; d < D; d++)
        for (int64_t i = doc_off[d]; i < doc_off[d + 1]; i++) m_dk[d * K + z[i]] += 1;
}

/* ------------------------------------------------------------------------ */
/* Phi-step: c_{k,v} ~ Pois(beta + n_{k,v}) for every entry (Eq. 9),        */
/* S_k = sum_v c_{k,v}; rows with S_k = 0 are redrawn (R-DEAD).              */
/* ------------------------------------------------------------------------ */

/* Pois(beta) over the positions 0..len-1 whose n is zero, by geometric
   skip-ahead.  n_at(pos) reads n; out(pos) receives the value.  Counters:
   (c0, h, sweep, tag<<28 | aux) for hit h = 0, 1, ... */
static void beta_field(const or_ctx *c, uint64_t seed, uint32_t sweep, uint32_t tag, uint32_t aux,
                       uint32_t c0, int64_t len, const int32_t *n, int64_t n_stride,
                       uint32_t *out, int64_t out_stride)
{
    int64_t pos = -1;
    uint32_t h = 0;
    for (;;) {
        uint32_t x[4];
        draw4(seed, c0, h, sweep, tag, aux, x);
        h++;
        int32_t g = geo_gap(c, x[0]);
        if (g < 0) {                       /* no hit among the next LG positions */
            pos += OR_LG;
            if (pos >= len - 1) break;
            continue;
        }
        pos += (int64_t)g + 1;
        if (pos >= len) break;
        if (n[pos * n_stride] == 0) out[pos * out_stride] = (uint32_t)alias_draw(&c->ztp, x[1], x[2]);
    }
}

/* Word v's entries c_{k,v}, k = 0..K-1 (its row of c_vk, zeroed first). */
static void phi_word(const or_ctx *c, const int32_t *n_vk, int32_t K, int32_t v,
                     uint64_t seed, uint32_t sweep, uint32_t *c_vk)
{
    const int32_t *nv = n_vk + (int64_t)v * K;
    uint32_t *cv = c_vk + (int64_t)v * K;
    memset(cv, 0, sizeof(uint32_t) * (size_t)K);
    for (int32_t k = 0; k < K; k++) {
        if (nv[k] == 0) continue;
        uint32_t x[4];
        draw4(seed, (uint32_t)v, (uint32_t)k, sweep, OR_TAG_POIS, 0, x);
        cv[k] = or_draw_entry(c, nv[k], x[0], x[1]);
    }
    beta_field(c, seed, sweep, OR_TAG_BETA, 0, (uint32_t)v, K, nv, 1, cv, 1);
}

/* Row k of Phi redrawn until its sum is nonzero (R-DEAD); returns the sum,
   or 0 if it stayed zero for OR_MAX_REDRAW attempts. */
static int64_t phi_redraw_row(const or_ctx *c, const int32_t *n_vk, int32_t K, int32_t V, int32_t k,
                              uint64_t seed, uint32_t sweep, uint32_t *c_vk);

int32_t or_phi_draw(const or_ctx *c, const int32_t *n_vk, int32_t K, int32_t V,
                    uint64_t seed, uint32_t sweep, uint32_t *c_vk, int64_t *S, int32_t *dead_rows)
{
    for (int32_t v = 0; v < V; v++) phi_word(c, n_vk, K, v, seed, sweep, c_vk);
    for (int32_t k = 0; k < K; k++) {
        S[k] = 0;
        for (int32_t v = 0; v < V; v++) S[k] += c_vk[(int64_t)v * K + k];
    }
    int32_t dead = 0;
    for (int32_t k = 0; k < K; k++) {
        if (S[k] != 0) continue;
        dead++;
        S[k] = phi_redraw_row(c, n_vk, K, V, k, seed, sweep, c_vk);
        if (S[k] == 0) return -1;
    }
    *dead_rows = dead;
    return 0;
}

static int64_t phi_redraw_row(const or_ctx *c, const int32_t *n_vk, int32_t K, int32_t V, int32_t k,
                              uint64_t seed, uint32_t sweep, uint32_t *c_vk)
{
    {
        uint32_t a;
        for (a = 1; a <= OR_MAX_REDRAW; a++) {
            for (int32_t v = 0; v < V; v++) {
                int32_t l = n_vk[(int64_t)v * K + k];
                uint32_t val = 0;
                if (l > 0) {
                    uint32_t x[4];
                    draw4(seed, (uint32_t)v, (uint32_t)k, sweep, OR_TAG_REDRAW_POIS, a, x);
                    val = or_draw_entry(c, l, x[0], x[1]);
                }
                c_vk[(int64_t)v * K + k] = val;
            }
            beta_field(c, seed, sweep, OR_TAG_REDRAW_BETA, a, (uint32_t)k, V,
                       n_vk + k, K, c_vk + k, K);
            int64_t s = 0;
            for (int32_t v = 0; v < V; v++) s += c_vk[(int64_t)v * K + k];
            if (s > 0) return s;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-word tables for the z-step ("Efficient sampling of z"): the word's   */
/* nonzero phi entries in ascending topic order, their fixed-point weights  */
/* q, the alpha-part weights a = q * alpha (in 2^-16 units), sigma_a = A and */
/* the alias table over a.  phi32 = fp32(c / S) is the exported Phi.        */
/* ------------------------------------------------------------------------ */
/* Word v's tables; phi64, a and al are scratch of K entries. */
static void word_table(const uint32_t *c_vk, const int64_t *S, const float *alpha, int32_t K, int32_t v,
                       int32_t *ncol, int16_t *topic, uint32_t *q, uint64_t *A,
                       uint32_t *athr, int16_t *atopic, float *phi32, double *phi64, uint64_t *a, int32_t *al)
{
    {
        const uint32_t *cv = c_vk + (int64_t)v * K;
        int64_t base = (int64_t)v * K;
        int32_t n = 0;
        double phimax = 0.0;
        for (int32_t k = 0; k < K; k++) {
            if (cv[k] == 0) continue;
            double p = (double)cv[k] / (double)S[k];   /* phi_{k,v} = c_{k,v} / S_k */
            topic[base + n] = (int16_t)k;
            phi64[n] = p;
            phi32[base + n] = (float)p;
            if (p > phimax) phimax = p;
            n++;
        }
        ncol[v] = n;
        if (n == 0) { A[v] = 0; return; }
        int e;
        frexp(phimax, &e);                 /* phimax = f 2^e, f in [1/2, 1) */
        uint64_t tot = 0;
        for (int32_t j = 0; j < n; j++) {
            double qq = floor(ldexp(phi64[j], 24 - e) + 0.5);
            uint32_t qj = qq < 1.0 ? 1u : (uint32_t)qq;
            q[base + j] = qj;
            int32_t k = topic[base + j];
            a[j] = (uint64_t)floor(ldexp((double)qj * (double)alpha[k], OR_FRAC_BITS) + 0.5);
            tot += a[j];
        }
        A[v] = tot;                        /* sigma_a in units of 2^-16 q */
        or_vose(a, n, athr + base, al);
        for (int32_t j = 0; j < n; j++) atopic[base + j] = topic[base + al[j]];
    }
}

void or_word_tables(const uint32_t *c_vk, const int64_t *S, const float *alpha, int32_t K, int32_t V,
                    int32_t *ncol, int16_t *topic, uint32_t *q, uint64_t *A,
                    uint32_t *athr, int16_t *atopic, float *phi32)
{
    double *phi64 = (double *)malloc(sizeof(double) * (size_t)K);
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)K);
    int32_t *al = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    for (int32_t v = 0; v < V; v++)
        word_table(c_vk, S, alpha, K, v, ncol, topic, q, A, athr, atopic, phi32, phi64, a, al);
    free(phi64); free(a); free(al);
}

/* ------------------------------------------------------------------------ */
/* z-step (Algorithm 2, second bullet): every document in turn, every token */
/* in order; p(z_i = k) proportional to phi_{k,v}(alpha_k + m^{-i}_{d,k}),  */
/* split into a (alpha part, alias table) and b (m part, iterated).         */
/* stats[0] += tokens, stats[1] += a-branch draws, stats[2] += sum over      */
/* tokens of min(K_d, K_v), stats[3] += zero-mass tokens kept, stats[4] +=   */
/* |J| (topics nonzero in both m^{-i} and the column), stats[5] += tokens    */
/* with K_d < K_v.                                                           */
/* ------------------------------------------------------------------------ */
/* One token's step (Algorithm 2, second bullet): remove token i from the
 * document counts m (K_d = *kd nonzero entries), draw its topic from
 * p(k) proportional to phi_{k,v}(alpha_k + m^{-i}_k) in the exact integer
 * form of "Efficient sampling of z", add it back.  Returns the new topic, or
 * -1 if the search ran past the total (which cannot happen). */
static int32_t z_token(int64_t i, int32_t v, int32_t kold, int64_t *m, int64_t *kd, int32_t K,
                       const int32_t *ncol, const int16_t *topic, const uint32_t *q, const uint64_t *A,
                       const uint32_t *athr, const int16_t *atopic,
                       uint64_t seed, uint32_t sweep, int64_t index_base, int64_t *stats)
{
    if (--m[kold] == 0) (*kd)--;           /* m^{-i}: remove token i */
    int64_t base = (int64_t)v * K;
    int32_t nv = ncol[v];
    /* sigma_b = sum_k q_{k,v} m^{-i}_{d,k}; every term is exact */
    uint64_t B = 0;
    for (int32_t j = 0; j < nv; j++) {
        B += (uint64_t)q[base + j] * (uint64_t)m[topic[base + j]];
        if (m[topic[base + j]] > 0) stats[4]++;
    }
    if (*kd < nv) stats[5]++;
    uint64_t T = A[v] + (B << OR_FRAC_BITS);
    int32_t knew = kold;
    uint64_t t = (uint64_t)(index_base + i);
    uint32_t x[4];
    draw4(seed, (uint32_t)t, (uint32_t)(t >> 32), sweep, OR_TAG_Z, 0, x);
    if (T == 0) {
        stats[3]++;
    } else {
        uint64_t U = ((uint64_t)x[0] << 32) | x[1];
        uint64_t r = (uint64_t)(((unsigned __int128)U * T) >> 64);   /* u (sigma_a + sigma_b) */
        if (r < A[v]) {
            uint32_t s = scale32(x[2], (uint32_t)nv);
            knew = x[3] < athr[base + s] ? topic[base + s] : atopic[base + s];
            stats[1]++;
        } else {
            uint64_t rb = (r - A[v]) >> OR_FRAC_BITS;
            uint64_t C = 0;
            knew = -1;
            for (int32_t j = 0; j < nv; j++) {
                C += (uint64_t)q[base + j] * (uint64_t)m[topic[base + j]];
                if (rb < C) { knew = topic[base + j]; break; }
            }
            if (knew < 0) return -1;           /* cannot happen: rb < B */
        }
    }
    stats[0]++;
    stats[2] += *kd < nv ? *kd : nv;
    if (m[knew]++ == 0) (*kd)++;
    return knew;
}

/* Document d's tokens in order (in slices of slice_len with stale counts
   when slice_len > 0 and the document is longer); m0 and m are scratch of K
   entries. */
static int32_t z_doc(int64_t d, const int64_t *doc_off, const int32_t *w, int16_t *z, int32_t K,
                     const int32_t *ncol, const int16_t *topic, const uint32_t *q, const uint64_t *A,
                     const uint32_t *athr, const int16_t *atopic, uint64_t seed, uint32_t sweep,
                     int64_t index_base, int64_t slice_len, int64_t *stats, int64_t *m0, int64_t *m)
{
    memset(m0, 0, sizeof(int64_t) * (size_t)K);
    int64_t kd0 = 0;                    /* number of nonzero m_{d,k} */
    for (int64_t i = doc_off[d]; i < doc_off[d + 1]; i++)
        if (m0[z[i]]++ == 0) kd0++;
    int64_t len = doc_off[d + 1] - doc_off[d];
    int64_t step = (slice_len > 0 && len > slice_len) ? slice_len : len;
    for (int64_t a = doc_off[d]; a < doc_off[d + 1]; a += step) {
        memcpy(m, m0, sizeof(int64_t) * (size_t)K);
        int64_t kd = kd0;
        int64_t b = a + step < doc_off[d + 1] ? a + step : doc_off[d + 1];
        for (int64_t i = a; i < b; i++) {
            int32_t knew = z_token(i, w[i], z[i], m, &kd, K, ncol, topic, q, A, athr, atopic,
                                   seed, sweep, index_base, stats);
            if (knew < 0) return -1;
            z[i] = (int16_t)knew;
        }
    }
    return 0;
}

int32_t or_z_step(const int64_t *doc_off, int64_t D, const int32_t *w, int16_t *z, int32_t K, int32_t V,
                  const int32_t *ncol, const int16_t *topic, const uint32_t *q, const uint64_t *A,
                  const uint32_t *athr, const int16_t *atopic,
                  uint64_t seed, uint32_t sweep, int64_t index_base, int64_t *stats)
{
    return or_z_step_sliced(doc_off, D, w, z, K, V, ncol, topic, q, A, athr, atopic, seed, sweep, index_base, 0, stats);
}

/* The z-step with long documents split into concurrent slices (a different
 * sampler from Algorithm 2, outside the paper: within a document, AD-LDA's
 * stale counts).  A document longer than slice_len tokens is cut into slices
 * of slice_len tokens; each slice starts from m0, the document's counts at the
 * start of the pass, and updates only its own copy, in position order.  With
 * slice_len = 0, or no document longer than it, this is Algorithm 2 exactly. */
int32_t or_z_step_sliced(const int64_t *doc_off, int64_t D, const int32_t *w, int16_t *z, int32_t K, int32_t V,
                         const int32_t *ncol, const int16_t *topic, const uint32_t *q, const uint64_t *A,
                         const uint32_t *athr, const int16_t *atopic,
                         uint64_t seed, uint32_t sweep, int64_t index_base, int64_t slice_len, int64_t *stats)
{
    (void)V;
    int64_t *m0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    int64_t *m = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    int32_t rc = 0;
    for (int64_t d = 0; d < D && rc == 0; d++)
        rc = z_doc(d, doc_off, w, z, K, ncol, topic, q, A, athr, atopic, seed, sweep, index_base, slice_len,
                   stats, m0, m);
    free(m0);
    free(m);
    return rc;
}

/* ------------------------------------------------------------------ Dirichlet Phi (Algorithm 1)
 * The partially collapsed sampler the Polya urn approximates (Algorithm 1,
 * "Efficient sampling of Phi"): phi_k ~ Dir(n_k + beta), drawn through the
 * Gamma representation gamma_{k,v} ~ G(beta + n_{k,v}, 1), phi_{k,v} =
 * gamma_{k,v} / sum_v gamma_{k,v}, with Gammas by Marsaglia and Tsang (2000).
 * Readings (the paper fixes none of these):
 *   R-GAMMA  float arithmetic, each operation rounded to float; normals from
 *            the rounded-normal table (R-GAUSS), uniforms with 23 bits
 *            u = (2 floor(x / 2^9) + 1) 2^-24; Philox counter (v, k, sweep,
 *            7 << 28 | attempt) per attempt, (v, k, sweep, 8 << 28) for the
 *            boost u^(1/a) of shapes a < 1 (Marsaglia and Tsang, Section 6);
 *            log and exp are this file's own (below), not libm's.
 *   R-DIRSUM S_k = sum over chunks of 256 words, in ascending order, of the
 *            chunk's sum of gamma_{k,v} in ascending v, all in double.
 *   R-DIRFIX phi_{k,v} = gamma_{k,v} * (1 / S_k) in double; q as in R-FIX
 *            but without the floor at 1: entries whose q rounds to 0 (phi
 *            below 2^(e-25), the column maximum lying in [2^(e-1), 2^e), so
 *            below 2^-24 of the maximum) leave the column.  This is the
 *            Dirichlet counterpart of Phi's sparsity; it drops at most
 *            K 2^-24 of a column's largest entry.
 */
#define OR_TAG_GAMMA 7u
#define OR_TAG_GAMMA_BOOST 8u
#define OR_DIR_CHUNK 256
#define OR_MAX_GAMMA_TRY (1u << 16)

static float f_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_f(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* ln x for finite x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)];
 * ln m = 2 atanh(s), s = (m - 1) / (m + 1), |s| <= 0.1716, by its series to
 * s^9 (the next term is below 2^-28 relative); ln 2 split Cody-Waite style. */
float or_logf(float x)
{
    int32_t e = 0;
    uint32_t b = bits_f(x);
    if (b < 0x00800000u) { x = x * 16777216.0f; b = bits_f(x); e = -24; }   /* subnormal: scale by 2^24 */
    e += (int32_t)(b >> 23) - 127;
    float m = f_bits((b & 0x007FFFFFu) | 0x3F800000u);                     /* [1, 2) */
    if (m > 1.41421354f) { m = m * 0.5f; e += 1; }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float poly = s * (2.0f + s2 * (0.666666687f + s2 * (0.400000006f + s2 * (0.285714298f + s2 * 0.222222224f))));
    float ef = (float)e;
    return ef * 0.693359375f + (ef * -2.12194442e-4f + poly);
}

/* e^x for x <= 88: x = k ln 2 + r, |r| <= ln 2 / 2, e^r by its Taylor series
 * to r^7 (next term below 2^-27 relative), scaled by 2^k; 0 below -104. */
float or_expf(float x)
{
    if (x < -104.0f) return 0.0f;
    float kf = floorf(x * 1.44269502f + 0.5f);
    int32_t k = (int32_t)kf;
    float r = (x - kf * 0.693359375f) - kf * -2.12194442e-4f;
    float p = 1.0f + r * (1.0f + r * (0.5f + r * (0.166666672f + r * (0.0416666679f + r * (0.00833333377f +
              r * (0.00138888892f + r * 0.000198412701f))))));
    if (k >= -126) return p * f_bits((uint32_t)(k + 127) << 23);
    return (p * f_bits((uint32_t)(k + 64 + 127) << 23)) * f_bits((uint32_t)(127 - 64) << 23);
}

static float unif23(uint32_t x)
{
    return (float)(2u * (x >> 9) + 1u) * 5.96046448e-08f;   /* (2 floor(x/2^9) + 1) 2^-24 */
}

/* gamma ~ G(a, 1), a > 0 (R-GAMMA).  *err is set when no attempt in
 * OR_MAX_GAMMA_TRY was accepted (probability below 0.05^65536). */
float or_gamma_draw(const or_ctx *c, float a, uint64_t seed, uint32_t v, uint32_t k, uint32_t sweep, int32_t *err)
{
    float sh = a < 1.0f ? a + 1.0f : a;
    float d = sh - 0.333333343f;
    float cc = 1.0f / sqrtf(9.0f * d);
    for (uint32_t t = 0; t < OR_MAX_GAMMA_TRY; t++) {
        uint32_t x[4];
        draw4(seed, v, k, sweep, OR_TAG_GAMMA, t, x);
        float g = (float)or_gauss_draw(c, x[0], x[1]);
        float y = 1.0f + cc * g;
        if (y <= 0.0f) continue;
        float v3 = (y * y) * y;
        float u = unif23(x[2]);
        float g2 = g * g;
        if (u < 1.0f - 0.0331f * (g2 * g2) || or_logf(u) < 0.5f * g2 + d * ((1.0f - v3) + or_logf(v3))) {
            float r = d * v3;
            if (a < 1.0f) {
                uint32_t xb[4];
                draw4(seed, v, k, sweep, OR_TAG_GAMMA_BOOST, 0, xb);
                r = r * or_expf(or_logf(unif23(xb[0])) / a);
            }
            return r;
        }
    }
    *err = 1;
    return 0.0f;
}

/* Algorithm 1, first bullet: gamma_{k,v} ~ G(beta + n_{k,v}, 1) for every
 * entry (g_vk[v*K + k], shape beta + n rounded to float) and S_k (R-DIRSUM). */
int32_t or_phi_draw_dir(const or_ctx *c, const int32_t *n_vk, int32_t K, int32_t V, uint64_t seed, uint32_t sweep,
                        float *g_vk, double *S)
{
    int32_t err = 0;
    float bf = (float)c->beta;
    for (int32_t v = 0; v < V; v++)
        for (int32_t k = 0; k < K; k++) {
            int64_t o = (int64_t)v * K + k;
            g_vk[o] = or_gamma_draw(c, bf + (float)n_vk[o], seed, (uint32_t)v, (uint32_t)k, sweep, &err);
        }
    for (int32_t k = 0; k < K; k++) {
        double tot = 0.0;
        for (int32_t v0 = 0; v0 < V; v0 += OR_DIR_CHUNK) {
            double part = 0.0;
            for (int32_t v = v0; v < V && v < v0 + OR_DIR_CHUNK; v++) part += (double)g_vk[(int64_t)v * K + k];
            tot += part;
        }
        S[k] = tot;
    }
    return err ? -1 : 0;
}

/* Per-word tables of the Dirichlet Phi (R-DIRFIX); the rest as or_word_tables. */
void or_word_tables_dir(const float *g_vk, const double *S, const float *alpha, int32_t K, int32_t V,
                        int32_t *ncol, int16_t *topic, uint32_t *q, uint64_t *A,
                        uint32_t *athr, int16_t *atopic, float *phi32)
{
    double *inv = (double *)malloc(sizeof(double) * (size_t)K);
    double *p = (double *)malloc(sizeof(double) * (size_t)K);
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)K);
    int32_t *al = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    for (int32_t k = 0; k < K; k++) inv[k] = S[k] > 0.0 ? 1.0 / S[k] : 0.0;   /* a row of underflows: phi_k = 0 */
    for (int32_t v = 0; v < V; v++) {
        int64_t base = (int64_t)v * K;
        double phimax = 0.0;
        for (int32_t k = 0; k < K; k++) {
            p[k] = (double)g_vk[base + k] * inv[k];
            if (p[k] > phimax) phimax = p[k];
        }
        int32_t n = 0;
        uint64_t tot = 0;
        if (phimax > 0.0) {
            int e;
            frexp(phimax, &e);
            for (int32_t k = 0; k < K; k++) {
                double qq = floor(ldexp(p[k], 24 - e) + 0.5);
                if (qq < 1.0) continue;            /* below 2^-25 of the column maximum */
                topic[base + n] = (int16_t)k;
                q[base + n] = (uint32_t)qq;
                phi32[base + n] = (float)p[k];
                a[n] = (uint64_t)floor(ldexp(qq * (double)alpha[k], OR_FRAC_BITS) + 0.5);
                tot += a[n];
                n++;
            }
        }
        ncol[v] = n;
        A[v] = tot;
        if (n == 0) continue;
        or_vose(a, n, athr + base, al);
        for (int32_t j = 0; j < n; j++) atopic[base + j] = topic[base + al[j]];
    }
    free(inv); free(p); free(a); free(al);
}

/* ------------------------------------------------------------------ log posterior
 * Diagnostic of the experiments (Section 5, the log-posterior trace plots):
 * the collapsed log joint of the topic indicators and the words, with Theta
 * and Phi integrated out of the Dirichlet-multinomial LDA model (notation
 * table, Section 1):
 *
 *   log p(w, z | alpha, beta)
 *     = sum_d [ lgamma(sum_k alpha_k) - lgamma(sum_k alpha_k + N_d)
 *               + sum_k ( lgamma(alpha_k + m_{d,k}) - lgamma(alpha_k) ) ]
 *     + sum_k [ lgamma(V beta) - lgamma(V beta + n_k)
 *               + sum_v ( lgamma(beta + n_{k,v}) - lgamma(beta) ) ],
 *
 * n_k = sum_v n_{k,v}.  As a function of z it is the unnormalised marginal
 * posterior p(z | w).  out[0] = total, out[1] = the document sum, out[2] =
 * the topic sum.  Terms with a zero count are exactly zero and skipped; every
 * sum runs in index order in double.  Returns -1 on allocation failure. */
int32_t or_log_posterior(const int64_t *doc_off, int64_t D, const int32_t *w, const int16_t *z,
                         int32_t K, int32_t V, const float *alpha, double beta, double out[3])
{
    int64_t N = doc_off[D];
    double asum = 0.0;
    for (int32_t k = 0; k < K; k++) asum += (double)alpha[k];
    int32_t *m = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    int32_t *n = (int32_t *)malloc(sizeof(int32_t) * (size_t)K * (size_t)V);
    int64_t *nk = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    if (!m || !n || !nk) { free(m); free(n); free(nk); return -1; }
    double docs = 0.0;
    for (int64_t d = 0; d < D; d++) {
        memset(m, 0, sizeof(int32_t) * (size_t)K);
        for (int64_t i = doc_off[d]; i < doc_off[d + 1]; i++) m[z[i]]++;
        double t = lgamma(asum) - lgamma(asum + (double)(doc_off[d + 1] - doc_off[d]));
        for (int32_t k = 0; k < K; k++)
            if (m[k] > 0) t += lgamma((double)alpha[k] + (double)m[k]) - lgamma((double)alpha[k]);
        docs += t;
    }
    or_count_n(N, w, z, K, V, n);
    double topics = 0.0;
    for (int32_t k = 0; k < K; k++) {
        double t = 0.0;
        for (int32_t v = 0; v < V; v++) {
            int32_t c = n[(int64_t)v * K + k];
            if (c > 0) { t += lgamma(beta + (double)c) - lgamma(beta); nk[k] += c; }
        }
        topics += t + lgamma((double)V * beta) - lgamma((double)V * beta + (double)nk[k]);
    }
    free(m); free(n); free(nk);
    out[0] = docs + topics;
    out[1] = docs;
    out[2] = topics;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The same steps over several host threads.  Algorithm 2 resamples the      */
/* documents independently ("in parallel for d"), and the Phi-step draws     */
/* every word's entries independently; here each thread runs the per-word    */
/* and per-document steps above on whole words and documents, taken from a   */
/* shared counter.  Every draw is keyed by (token | word, topic, sweep) and  */
/* every count and sum is an exact integer, so the results are bit for bit   */
/* the single-threaded functions' whatever the thread count and schedule.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int kind;                     /* 0 counts, 1 Phi rows of words, 2 dead-row redraws, 3 tables, 4 documents */
    int64_t total, chunk;         /* work items and how many a thread takes at once */
    int64_t next;                 /* shared counter (atomic) */
    int32_t err;                  /* set (atomic) by a failing item */
    /* arguments */
    const or_ctx *c;
    int64_t N; int32_t K, V;
    const int32_t *w; int16_t *z; const int64_t *doc_off;
    const int32_t *n_vk; uint32_t *c_vk; int64_t *S; const int32_t *dead_k;
    const float *alpha; int32_t *ncol; int16_t *topic; uint32_t *q; uint64_t *A; uint32_t *athr;
    int16_t *atopic; float *phi32;
    uint64_t seed; uint32_t sweep; int64_t index_base;
    int64_t stats[6];             /* summed (atomic) from the threads' own counters */
} mt_job;

static void *mt_worker(void *arg)
{
    mt_job *j = (mt_job *)arg;
    const int32_t K = j->K;
    double *phi64 = NULL; uint64_t *a = NULL; int32_t *al = NULL; int64_t *m0 = NULL, *m = NULL;
    if (j->kind == 3) {
        phi64 = (double *)malloc(sizeof(double) * (size_t)K);
        a = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)K);
        al = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
        if (!phi64 || !a || !al) { __atomic_store_n(&j->err, 1, __ATOMIC_RELAXED); goto out; }
    }
    if (j->kind == 4) {
        m0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
        m = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
        if (!m0 || !m) { __atomic_store_n(&j->err, 1, __ATOMIC_RELAXED); goto out; }
    }
    int64_t st[6] = {0, 0, 0, 0, 0, 0};
    for (;;) {
        int64_t lo = __atomic_fetch_add(&j->next, j->chunk, __ATOMIC_RELAXED);
        if (lo >= j->total) break;
        int64_t hi = lo + j->chunk < j->total ? lo + j->chunk : j->total;
        for (int64_t i = lo; i < hi; i++) {
            switch (j->kind) {
            case 0:
                __atomic_fetch_add(&((int32_t *)j->n_vk)[(int64_t)j->w[i] * K + j->z[i]], 1, __ATOMIC_RELAXED);
                break;
            case 1:
                phi_word(j->c, j->n_vk, K, (int32_t)i, j->seed, j->sweep, j->c_vk);
                break;
            case 2: {
                int32_t k = j->dead_k[i];
                j->S[k] = phi_redraw_row(j->c, j->n_vk, K, j->V, k, j->seed, j->sweep, j->c_vk);
                if (j->S[k] == 0) __atomic_store_n(&j->err, 1, __ATOMIC_RELAXED);
                break;
            }
            case 3:
                word_table(j->c_vk, j->S, j->alpha, K, (int32_t)i, j->ncol, j->topic, j->q, j->A, j->athr,
                           j->atopic, j->phi32, phi64, a, al);
                break;
            default:
                if (z_doc(i, j->doc_off, j->w, j->z, K, j->ncol, j->topic, j->q, j->A, j->athr, j->atopic,
                          j->seed, j->sweep, j->index_base, 0, st, m0, m) != 0)
                    __atomic_store_n(&j->err, 1, __ATOMIC_RELAXED);
            }
        }
    }
    for (int t = 0; t < 6; t++) __atomic_fetch_add(&j->stats[t], st[t], __ATOMIC_RELAXED);
out:
    free(phi64); free(a); free(al); free(m0); free(m);
    return NULL;
}

/* Runs job j on n_threads threads (the calling one included); 0 on success. */
static int32_t mt_run(mt_job *j, int32_t n_threads)
{
    if (n_threads < 1) n_threads = 1;
    j->next = 0;
    j->err = 0;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    if (!th) return -1;
    int32_t started = 0;
    for (int32_t t = 1; t < n_threads; t++)
        if (pthread_create(&th[t], NULL, mt_worker, j) == 0) started = t;
        else break;
    mt_worker(j);
    for (int32_t t = 1; t <= started; t++) pthread_join(th[t], NULL);
    free(th);
    return j->err ? -1 : 0;
}

void or_count_n_mt(int64_t N, const int32_t *w, const int16_t *z, int32_t K, int32_t V, int32_t *n_vk,
                   int32_t n_threads)
{
    memset(n_vk, 0, sizeof(int32_t) * (size_t)K * (size_t)V);
    mt_job j;
    memset(&j, 0, sizeof j);
    j.kind = 0; j.total = N; j.chunk = 1 << 16; j.K = K; j.V = V; j.w = w; j.z = (int16_t *)z; j.n_vk = n_vk;
    mt_run(&j, n_threads);
}

int32_t or_phi_draw_mt(const or_ctx *c, const int32_t *n_vk, int32_t K, int32_t V, uint64_t seed, uint32_t sweep,
                       uint32_t *c_vk, int64_t *S, int32_t *dead_rows, int32_t n_threads)
{
    mt_job j;
    memset(&j, 0, sizeof j);
    j.kind = 1; j.total = V; j.chunk = 16; j.c = c; j.K = K; j.V = V; j.n_vk = n_vk; j.c_vk = c_vk;
    j.seed = seed; j.sweep = sweep;
    if (mt_run(&j, n_threads) != 0) return -1;
    for (int32_t k = 0; k < K; k++) S[k] = 0;
    for (int32_t v = 0; v < V; v++)
        for (int32_t k = 0; k < K; k++) S[k] += c_vk[(int64_t)v * K + k];
    int32_t *dead = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    if (!dead) return -1;
    int32_t nd = 0;
    for (int32_t k = 0; k < K; k++)
        if (S[k] == 0) dead[nd++] = k;
    j.kind = 2; j.total = nd; j.chunk = 1; j.S = S; j.dead_k = dead;
    int32_t rc = mt_run(&j, n_threads);
    free(dead);
    if (rc != 0) return -1;
    *dead_rows = nd;
    return 0;
}

void or_word_tables_mt(const uint32_t *c_vk, const int64_t *S, const float *alpha, int32_t K, int32_t V,
                       int32_t *ncol, int16_t *topic, uint32_t *q, uint64_t *A,
                       uint32_t *athr, int16_t *atopic, float *phi32, int32_t n_threads)
{
    mt_job j;
    memset(&j, 0, sizeof j);
    j.kind = 3; j.total = V; j.chunk = 64; j.K = K; j.V = V; j.c_vk = (uint32_t *)c_vk; j.S = (int64_t *)S;
    j.alpha = alpha; j.ncol = ncol; j.topic = topic; j.q = q; j.A = A; j.athr = athr; j.atopic = atopic;
    j.phi32 = phi32;
    mt_run(&j, n_threads);
}

int32_t or_z_step_mt(const int64_t *doc_off, int64_t D, const int32_t *w, int16_t *z, int32_t K, int32_t V,
                     const int32_t *ncol, const int16_t *topic, const uint32_t *q, const uint64_t *A,
                     const uint32_t *athr, const int16_t *atopic,
                     uint64_t seed, uint32_t sweep, int64_t index_base, int64_t *stats, int32_t n_threads)
{
    mt_job j;
    memset(&j, 0, sizeof j);
    j.kind = 4; j.total = D; j.chunk = 16; j.K = K; j.V = V; j.doc_off = doc_off; j.w = w; j.z = z;
    j.ncol = (int32_t *)ncol; j.topic = (int16_t *)topic; j.q = (uint32_t *)q; j.A = (uint64_t *)A;
    j.athr = (uint32_t *)athr; j.atopic = (int16_t *)atopic; j.seed = seed; j.sweep = sweep;
    j.index_base = index_base;
    int32_t rc = mt_run(&j, n_threads);
    for (int t = 0; t < 6; t++) stats[t] += j.stats[t];
    return rc;
}
