/*
 * pulda_oracle.h -- declarations of the CPU oracle (test infrastructure only;
 * see pulda_oracle.c).  Not used by, and not visible to, the CUDA library.
 */
#ifndef PULDA_ORACLE_H
#define PULDA_ORACLE_H
#include <stdint.h>

#define OR_L 100                 /* alias tables for rates beta + l, l <= L ("Efficient sampling of Phi") */
#define OR_LG 1024               /* geometric-gap table length */
#define OR_GAUSS_CELLS 65536     /* equiprobable inverse-normal cells */
#define OR_GAUSS_TAIL_P 5.9604644775390625e-08 /* 2^-24: outer edge of the two tail cells */
#define OR_FRAC_BITS 16          /* alpha terms in units of 2^-16 */
#define OR_MAX_REDRAW (1u << 20) /* dead-row redraw attempts */

#define OR_TAG_INIT 1u
#define OR_TAG_POIS 2u
#define OR_TAG_BETA 3u
#define OR_TAG_REDRAW_POIS 4u
#define OR_TAG_REDRAW_BETA 5u
#define OR_TAG_Z 6u

typedef struct or_ctx or_ctx;

void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint64_t or_vose(const uint64_t *W, int32_t n, uint32_t *thr, int32_t *alias);
int32_t or_pois_weights(double lam, int32_t jmin, int32_t cap, int64_t *lo_out, uint64_t *W);
double or_norm_quantile(double p);
void or_gauss_table(double *Q);
void or_geo_table(double beta, uint32_t *thr);

or_ctx *or_ctx_new(float beta);
void or_ctx_free(or_ctx *c);
int32_t or_ctx_table(const or_ctx *c, int32_t which, int64_t *lo, uint32_t *thr, int32_t *alias);
void or_ctx_geo(const or_ctx *c, uint32_t *thr);
void or_ctx_gauss(const or_ctx *c, double *Q);
double or_gauss_draw(const or_ctx *c, uint32_t x0, uint32_t x1);
uint32_t or_draw_entry(const or_ctx *c, int64_t l, uint32_t x0, uint32_t x1);

void or_init_z(int64_t N, int32_t K, uint64_t seed, int64_t index_base, int16_t *z);
void or_count_n(int64_t N, const int32_t *w, const int16_t *z, int32_t K, int32_t V, int32_t *n_vk);
void or_doc_topic(const int64_t *doc_off, int64_t D, const int16_t *z, int32_t K, int32_t *m_dk);
int32_t or_phi_draw(const or_ctx *c, const int32_t *n_vk, int32_t K, int32_t V,
                    uint64_t seed, uint32_t sweep, uint32_t *c_vk, int64_t *S, int32_t *dead_rows);
void or_word_tables(const uint32_t *c_vk, const int64_t *S, const float *alpha, int32_t K, int32_t V,
                    int32_t *ncol, int16_t *topic, uint32_t *q, uint64_t *A,
                    uint32_t *athr, int16_t *atopic, float *phi32);
int32_t or_z_step(const int64_t *doc_off, int64_t D, const int32_t *w, int16_t *z, int32_t K, int32_t V,
                  const int32_t *ncol, const int16_t *topic, const uint32_t *q, const uint64_t *A,
                  const uint32_t *athr, const int16_t *atopic,
                  uint64_t seed, uint32_t sweep, int64_t index_base, int64_t *stats);
int32_t or_z_step_sliced(const int64_t *doc_off, int64_t D, const int32_t *w, int16_t *z, int32_t K, int32_t V,
                         const int32_t *ncol, const int16_t *topic, const uint32_t *q, const uint64_t *A,
                         const uint32_t *athr, const int16_t *atopic,
                         uint64_t seed, uint32_t sweep, int64_t index_base, int64_t slice_len, int64_t *stats);
int32_t or_log_posterior(const int64_t *doc_off, int64_t D, const int32_t *w, const int16_t *z,
                         int32_t K, int32_t V, const float *alpha, double beta, double out[3]);
float or_logf(float x);
float or_expf(float x);
float or_gamma_draw(const or_ctx *c, float a, uint64_t seed, uint32_t v, uint32_t k, uint32_t sweep, int32_t *err);
int32_t or_phi_draw_dir(const or_ctx *c, const int32_t *n_vk, int32_t K, int32_t V, uint64_t seed, uint32_t sweep,
                        float *g_vk, double *S);
void or_word_tables_dir(const float *g_vk, const double *S, const float *alpha, int32_t K, int32_t V,
                        int32_t *ncol, int16_t *topic, uint32_t *q, uint64_t *A,
                        uint32_t *athr, int16_t *atopic, float *phi32);
/* The same steps over n_threads host threads: results identical to the
   single-threaded functions (words, dead rows and documents are independent
   work items; every draw is keyed, every count exact). */
void or_count_n_mt(int64_t N, const int32_t *w, const int16_t *z, int32_t K, int32_t V, int32_t *n_vk,
                   int32_t n_threads);
int32_t or_phi_draw_mt(const or_ctx *c, const int32_t *n_vk, int32_t K, int32_t V, uint64_t seed, uint32_t sweep,
                       uint32_t *c_vk, int64_t *S, int32_t *dead_rows, int32_t n_threads);
void or_word_tables_mt(const uint32_t *c_vk, const int64_t *S, const float *alpha, int32_t K, int32_t V,
                       int32_t *ncol, int16_t *topic, uint32_t *q, uint64_t *A,
                       uint32_t *athr, int16_t *atopic, float *phi32, int32_t n_threads);
int32_t or_z_step_mt(const int64_t *doc_off, int64_t D, const int32_t *w, int16_t *z, int32_t K, int32_t V,
                     const int32_t *ncol, const int16_t *topic, const uint32_t *q, const uint64_t *A,
                     const uint32_t *athr, const int16_t *atopic,
                     uint64_t seed, uint32_t sweep, int64_t index_base, int64_t *stats, int32_t n_threads);
#endif
