/*
 * pulda.h -- C ABI of the GB300 Polya-urn partially collapsed LDA sampler
 * (Terenin, Magnusson, Jonsson, Draper, "Polya Urn Latent Dirichlet
 * Allocation: a doubly sparse massively parallel sampler", arXiv 1704.03581).
 *
 * One handle = one Markov chain on one GPU.  A sweep is Algorithm 2 of the
 * paper (Section 3): draw Phi with the Poisson Polya urn, then resample every
 * topic indicator z with the doubly sparse a/b split ("Efficient sampling of
 * z").  Every step runs in CUDA kernels; the host only validates arguments,
 * builds the fixed Poisson tables once, and copies data in and out.
 *
 * Conventions shared by every entry point
 *   - Pointers named *_host are host memory, *_dev device memory.  Inputs are
 *     read during the call and may be freed afterwards; the library keeps its
 *     own device copies.  Outputs are written into caller-allocated buffers of
 *     the stated size.
 *   - Every call returns a pulda_status.  On PULDA_ERR_INVALID the handle's
 *     state is unchanged; pulda_last_error() describes the problem.  A CUDA
 *     failure returns PULDA_ERR_CUDA and leaves the handle unusable except for
 *     pulda_free / pulda_last_error.
 *   - A handle is not thread safe: one host thread at a time.
 *   - Layouts: corpus in CSR form, word_ids[doc_offsets[d] .. doc_offsets[d+1])
 *     are document d's word ids in position order.  Topic ids are int16,
 *     0 <= k < K <= 16384.  Dense count outputs are row-major.
 *   - Random numbers: counter-based Philox4x32-10 keyed by the 64-bit seed,
 *     counter = (index_lo, index_hi, sweep, tag << 28 | aux); results depend
 *     only on (corpus, K, V, alpha, beta, seed, sweep count), never on launch
 *     shapes or timing.
 */
#ifndef PULDA_H
#define PULDA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PULDA_OK = 0,
    PULDA_ERR_INVALID = -1,     /* bad argument; state unchanged */
    PULDA_ERR_OOM = -2,         /* device allocation failed */
    PULDA_ERR_CUDA = -3,        /* a CUDA call or kernel failed */
    PULDA_ERR_TIMEOUT = -4,     /* a bounded wait expired */
    PULDA_ERR_DEGENERATE = -5,  /* a Phi row stayed all-zero after 2^20 redraws */
    PULDA_ERR_BUSY = -6         /* the server's slots or token budget are full */
} pulda_status;

typedef struct pulda_handle pulda_handle;

/* Launch options.  Zero-initialise and set what you need; NULL = defaults. */
typedef struct {
    void *stream;           /* cudaStream_t to run on; NULL = a stream the handle creates */
    int32_t zstep_path;     /* 0 = auto (iterate the smaller of the document's and the
                               word's nonzero topics), 1 = always iterate the word's Phi
                               column, 2 = iterate the document's topics whenever K <= 2048 */
    int32_t warps_per_block;/* warp-per-document z-step: warps per CTA, 1..4; 0 = 4, halved
                               while the CTA's shared memory would pass 160 KB */
    int32_t docs_per_warp;  /* z-step documents per warp: 0 = auto (one: measured faster at
                               every K), 1 = one, 4 = four (needs K <= 1024; falls back to
                               one when every word's dense q row does not fit 2 GB;
                               documents longer than 65,535 tokens still go one per warp,
                               the longest to CTAs as coop_min_len says); results are
                               identical */
    int32_t phi_mode;       /* 0 = Poisson Polya urn (Algorithm 2), 1 = Dirichlet (Algorithm 1:
                               phi_k ~ Dir(n_k + beta) through Gamma draws, entries below 2^-24
                               of their column's maximum dropped); the batched form takes 0 only */
    int32_t slice_len;      /* 0 = every document's tokens in order (Algorithm 2).  > 0: in the
                               corpus z-step (pulda_z_step, pulda_sweep) a document longer than
                               this is cut into slices of this many tokens, resampled
                               concurrently, each from the document's counts at the start of
                               the pass updated by its own tokens only -- stale counts across
                               slices, a different sampler from the paper's (AD-LDA's
                               approximation within a document).  Needs docs_per_warp 0 or 1;
                               fold-in, serving and the batched form ignore/reject it */
    int32_t coop_min_len;   /* corpus z-step and pulda_infer: a document at least this long is
                               resampled by the 4 warps of one CTA together, token by token
                               (its intersections split over 128 lanes), concurrently with the
                               other documents' one-warp kernel; results are identical.
                               0 = auto (documents longer than max(256, N / 8000) tokens,
                               N / 16000 beside four documents per warp: those that would
                               outlast the rest of the pass), -1 = never, > 0 = this length.
                               Not used with slice_len > 0; the batched form takes 0 or -1
                               (one warp per document); a server on the handle uses it for
                               requests (0 = requests of at least 1,024 tokens) */
    int32_t count_path;     /* how the Phi-step rebuilds n_{k,v}: 0 = shared-memory histogram of
                               each word's topics (the default, measured faster), 1 = radix sort
                               of every token's key w K + z and its runs (needs V K < 2^32; the
                               batched form takes 0); the counts are identical */
    int32_t batch_form;     /* batched form only: how a sweep is launched -- 0 = tuned (timed on
                               the first sweeps with the CTA sizes), 1 = six launches (a CUDA
                               graph), 2 = one persistent cooperative launch whose phases are
                               separated by grid barriers (every document one per warp; not
                               with coop_min_len > 0); the chains' results are identical */
    int32_t alias_layout;   /* how the per-word alias tables of the a part ("Efficient sampling
                               of z") are laid out for the z-step: 1 = a threshold array and an
                               alias-topic array beside the column's topics (two loads per
                               alias draw), 2 = also packed 8-byte slots {threshold, topic |
                               alias topic << 16} that the z-step reads instead (one load; 8
                               more bytes per entry of the table capacity K V); 0 = 1 on a
                               handle, tuned (timed on two sweeps each, after the launch
                               form) in the batched form; the tables' contents and every
                               result are identical */
    /* Device memory.  With alloc set, every device buffer the library takes
     * -- the handle's state in pulda_init, the temporaries of pulda_infer,
     * pulda_get_counts, pulda_get_phi and pulda_log_posterior, a server's
     * arenas and slot tables, a batch's tables -- comes from
     * alloc(bytes, stream, alloc_ctx) and goes back through
     * free(ptr, stream, alloc_ctx); `stream` is the handle's (or the
     * server's) cudaStream_t.  alloc must return device memory of the
     * handle's device aligned to 256 bytes, or NULL: the call then returns
     * PULDA_ERR_OOM after giving back everything it had taken (a misaligned
     * pointer is given back and reported as PULDA_ERR_CUDA).  A temporary
     * may be given back while work that reads it is still queued on
     * `stream`, so free must order the release after that work, as
     * cudaFreeAsync does (a stream-aware caching allocator does; otherwise
     * synchronise the stream first).  Both NULL = cudaMalloc for the state,
     * cudaMallocAsync for temporaries; only one set = PULDA_ERR_INVALID. */
    void *(*alloc)(size_t bytes, void *stream, void *alloc_ctx);
    void (*free)(void *ptr, void *stream, void *alloc_ctx);
    void *alloc_ctx;
} pulda_options;

/* Counters of the most recent z-step (and Phi-step), and running totals. */
typedef struct {
    int64_t tokens;          /* tokens resampled */
    int64_t a_branch;        /* draws taken from the alias table of the alpha part */
    int64_t sum_min;         /* sum over tokens of min(K_d^(m), K_v^(Phi)) (complexity theorem) */
    int64_t zero_mass;       /* tokens whose conditional had zero total mass (kept their topic) */
    int64_t dead_rows;       /* Phi rows redrawn because their Poisson counts summed to zero */
    int64_t nnz_phi;         /* nonzero entries of Phi */
    int64_t sweep;           /* sweep counter after the call */
    int64_t cum_tokens;      /* the z-step counters summed over every z-step since pulda_init */
    int64_t cum_a_branch;
    int64_t cum_sum_min;
    int64_t cum_zero_mass;
    int64_t sum_inter;       /* sum over tokens of |J|: topics nonzero in both m_d^{-i} and Phi's column */
    int64_t docside;         /* tokens with K_d < K_v (the document side is the smaller) */
    int64_t cum_sum_inter;
    int64_t cum_docside;
} pulda_sweep_stats;

/* pulda_init -- create a chain.
 * Model: LDA (Section 1, Figure "lda-dag", Table "notation") with symmetric or
 * per-topic alpha[K] and symmetric beta.  Topics start uniform (keyed by
 * (seed, token, sweep 0)); the paper does not prescribe an initialisation.
 *   word_ids_host   int32[N], N = doc_offsets_host[D]; every id in [0, V)
 *   doc_offsets_host int64[D+1], doc_offsets[0] = 0, nondecreasing
 *   K in [1, 16384], V >= 1, alpha[K] in (0, 256], beta in (0, 64]
 *   opt             may be NULL
 * Errors: PULDA_ERR_INVALID (bad sizes/ids/offsets/hyper-parameters; documents
 * longer than 2^22 tokens), PULDA_ERR_OOM, PULDA_ERR_CUDA. */
pulda_status pulda_init(pulda_handle **out, const int32_t *word_ids_host, const int64_t *doc_offsets_host,
                        int64_t D, int32_t K, int32_t V, const float *alpha_host, float beta,
                        uint64_t seed, const pulda_options *opt);

/* pulda_sweep -- n_sweeps iterations of Algorithm 2: for each, rebuild n from
 * z (notation table), draw Phi ~ PPU(n_k + beta) row by row (Definition "Poisson
 * Polya Urn", Eq. 9, "Efficient sampling of Phi"), then resample every z_{i,d}
 * proportional to phi_{k,v(i)}(alpha_k + m^{-i}_{d,k}) ("Efficient sampling of
 * z").  Asynchronous on the handle's stream; errors raised by kernels are
 * reported by the next pulda_sync.  Errors: PULDA_ERR_INVALID (n_sweeps < 0). */
pulda_status pulda_sweep(pulda_handle *h, int32_t n_sweeps);

/* pulda_phi_step / pulda_z_step -- the two halves of one sweep, for callers
 * that time or inspect them separately.  pulda_phi_step advances the sweep
 * counter and draws Phi for it; pulda_z_step resamples z with that Phi.
 * pulda_z_step before any pulda_phi_step returns PULDA_ERR_INVALID. */
pulda_status pulda_phi_step(pulda_handle *h);
pulda_status pulda_z_step(pulda_handle *h);

/* pulda_sync -- wait for the handle's stream and report device-side errors
 * (PULDA_ERR_DEGENERATE, PULDA_ERR_CUDA). */
pulda_status pulda_sync(pulda_handle *h);
/* pulda_sync_timeout -- as pulda_sync, but gives up after timeout_ms
 * milliseconds of waiting (polling the stream) and returns PULDA_ERR_TIMEOUT;
 * the work keeps running and a later pulda_sync waits for it.  Errors:
 * PULDA_ERR_INVALID (timeout_ms < 0), PULDA_ERR_TIMEOUT, as pulda_sync. */
pulda_status pulda_sync_timeout(pulda_handle *h, int32_t timeout_ms);

/* pulda_get_z -- copy z (int16[N], corpus order) to host / device memory. */
pulda_status pulda_get_z(pulda_handle *h, int16_t *z_host);
pulda_status pulda_get_z_dev(pulda_handle *h, int16_t *z_dev);

/* pulda_set_z -- replace z (int16[N], each in [0, K)) and set the sweep
 * counter; with the z and counter of an earlier pulda_get_z / pulda_stats this
 * resumes that chain exactly (n, m and Phi are functions of z and the keyed
 * random streams).  Errors: PULDA_ERR_INVALID (topic out of range). */
pulda_status pulda_set_z(pulda_handle *h, const int16_t *z_host, int64_t sweep);

/* pulda_get_counts -- exact counts from the current z (notation table):
 *   n_kv_host int32[K*V], n_kv[k*V + v] = #{i : z_i = k, w_i = v}, or NULL
 *   m_dk_host int32[D*K], m_dk[d*K + k] = #{i in d : z_i = k}, or NULL */
pulda_status pulda_get_counts(pulda_handle *h, int32_t *n_kv_host, int32_t *m_dk_host);

/* pulda_log_posterior -- the diagnostic of the paper's experiments (Section 5,
 * log-posterior trace plots): the collapsed log joint of the current topics,
 * Theta and Phi integrated out of Dirichlet-multinomial LDA,
 *   log p(w, z | alpha, beta)
 *     = sum_d [lgamma(A) - lgamma(A + N_d) + sum_k (lgamma(alpha_k + m_dk) - lgamma(alpha_k))]
 *     + sum_k [lgamma(V beta) - lgamma(V beta + n_k) + sum_v (lgamma(beta + n_kv) - lgamma(beta))],
 * A = sum_k alpha_k, n_k = sum_v n_kv; up to a constant it is log p(z | w).
 *   out_host double[3] = {total, document sum, topic sum}
 * beta is the handle's float beta widened to double.  The counts are rebuilt
 * from the current z on the GPU and every sum runs in a fixed order, so equal
 * topics give equal bits.  Synchronous; uses 8 (D + V + 257 K + 4099) bytes
 * of temporary device memory.  Errors: PULDA_ERR_INVALID (NULL out),
 * PULDA_ERR_CUDA. */
pulda_status pulda_log_posterior(pulda_handle *h, double *out_host);

/* pulda_get_phi -- the Phi drawn by the most recent Phi-step, sparse by word
 * (column-compressed): entries col_ptr[v] .. col_ptr[v+1]-1 hold the nonzero
 * phi_{k,v} = fp32(c_{k,v} / S_k) with topic ids in ascending order (Dirichlet
 * mode: fp32(gamma_{k,v} (1 / S_k)) over the entries kept).
 * Call with col_ptr/topic/phi NULL to query *nnz_inout; otherwise *nnz_inout
 * is the capacity of topic/phi on entry and the entry count on return.
 *   col_ptr_host int64[V+1], topic_host int16[nnz], phi_host float[nnz]
 * Errors: PULDA_ERR_INVALID (no Phi drawn yet, capacity too small). */
pulda_status pulda_get_phi(pulda_handle *h, int64_t *col_ptr_host, int16_t *topic_host, float *phi_host,
                           int64_t *nnz_inout);

/* pulda_get_word_tables -- the per-word z-step tables behind the current Phi
 * (for inspection and tests): Poisson counts c (uint32), row sums S (int64[K]),
 * fixed-point weights q (uint32), alpha-part masses A (uint64[V]) and the alias
 * table (threshold uint32, alias topic int16), laid out like pulda_get_phi.
 * In Dirichlet mode c holds the bits of the float Gamma draws and S the bits
 * of the double row sums.
 * Any output pointer may be NULL.  *nnz_inout as for pulda_get_phi. */
pulda_status pulda_get_word_tables(pulda_handle *h, int64_t *col_ptr_host, int16_t *topic_host,
                                   uint32_t *c_host, int64_t *S_host, uint32_t *q_host, uint64_t *A_host,
                                   uint32_t *athr_host, int16_t *atopic_host, int64_t *nnz_inout);

/* pulda_infer -- fold-in of new documents against the current Phi (Algorithm
 * 2's z-step with Phi held fixed): topics start uniform, keyed by (seed,
 * position in this call's token array, sweep 0), then n_sweeps z-steps with
 * sweep counters 1..n_sweeps.  The chain's own state is not changed.
 *   word_ids_host int32[N_new], doc_offsets_host int64[D_new+1]
 *   z_out_host int16[N_new] or NULL; m_out_host int32[D_new*K] or NULL
 * Errors: PULDA_ERR_INVALID (bad ids/offsets; no Phi drawn yet). */
pulda_status pulda_infer(pulda_handle *h, const int32_t *word_ids_host, const int64_t *doc_offsets_host,
                         int64_t D_new, int32_t n_sweeps, uint64_t seed, int16_t *z_out_host,
                         int32_t *m_out_host);

/* pulda_infer_noalloc -- pulda_infer for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant.
 * Serving processes that carve their device memory once at start-up,
 * memory-capped tenants of a shared GPU, and latency-critical loops that must
 * not stall on the allocator cannot call cudaMalloc (or anything that does);
 * pulda_infer allocates temporaries on every call, this call allocates
 * nothing.  The caller passes device buffers:
 *   word_ids_dev int32[N_new] (ids in [0, V)), doc_offsets_dev int64[D_new+1]
 *   (rising from 0 to N_new), z_out_dev int16[N_new] (the fold-in's topics,
 *   also its working state).
 * The results equal pulda_infer's with the same seed and n_sweeps.
 * The few bytes of scratch the z-step needs live in a fixed array of static
 * device memory (262,912 bytes, held by every GPU that loads the library until
 * the process exits), so D_new is limited to 65,536 documents per call; larger
 * D_new returns PULDA_ERR_INVALID.  The first call on each device looks up
 * that array's device address once; make that first call before any stream
 * capture.  The calling thread's current device must be the one the handle
 * was created on.  All calls on a device share the array: calls that overlap
 * on the GPU race and must be serialised by the caller.  The call waits for
 * the handle's stream before it returns.  Errors: PULDA_ERR_INVALID (limits,
 * NULL pointers, another current device, no Phi yet, bad ids or offsets --
 * checked on the device; the message names the first bad token or document),
 * PULDA_ERR_CUDA. */
pulda_status pulda_infer_noalloc(pulda_handle *h, const int32_t *word_ids_dev, const int64_t *doc_offsets_dev,
                                 int64_t D_new, int64_t N_new, int32_t n_sweeps, uint64_t seed,
                                 int16_t *z_out_dev);

/* ---------------------------------------------------------------- batches
 * Many independent chains advanced together (the batched form of Algorithm
 * 2): each chain is exactly the chain a handle with the same arguments would
 * run -- bit for bit -- but every kernel of a sweep runs once over all chains'
 * words and documents (longest first across chains), and the six launches of
 * a sweep are captured into one CUDA graph that is replayed every sweep.  The
 * z-step CTA size is chosen by timing the candidates on the first sweeps
 * (launch shapes never change results).  Chains may differ in D, N, K, V,
 * alpha, beta and seed; all share the batch's stream. */
typedef struct {
    const int32_t *word_ids_host;    /* int32[N] */
    const int64_t *doc_offsets_host; /* int64[D+1] */
    int64_t D;
    int32_t K, V;
    const float *alpha_host;         /* float[K] */
    float beta;
    uint64_t seed;
} pulda_chain_desc;

typedef struct pulda_batch pulda_batch;

/* pulda_batch_init -- validate and set up every chain as pulda_init would
 * (same limits and errors, reported with the chain's index).  opt->stream, if
 * set, is used for all chains; opt->warps_per_block in 1..8 fixes the z-step
 * CTA size instead of tuning it over {2, 4, 8}; opt->coop_min_len -1 keeps
 * every document on one warp, > 0 sends the documents at least that long (of
 * every chain) to the cooperative z-step, 0 sends those of at least
 * max(256, N / 8000) tokens (N = tokens of all chains), the single-chain rule;
 * docs_per_warp must be 0 or 1; batch_form picks the launch form and
 * alias_layout the alias tables' layout (see pulda_options).  Tuning times
 * each CTA size on two real sweeps (in order, then in reverse), together with
 * the one-launch form when no document goes to cooperative CTAs, then (with
 * alias_layout 0) the best of them with each alias layout on two sweeps each:
 * it ends after sweep 12 (10 without the one-launch form, 8 without the
 * layouts); every chain's tables then carry the packed slots (8 bytes per
 * entry of its K V capacity) unless alias_layout is 1. */
pulda_status pulda_batch_init(pulda_batch **out, const pulda_chain_desc *chains, int32_t n_chains,
                              const pulda_options *opt);
/* pulda_batch_sweep -- n_sweeps sweeps of every chain (asynchronous, except
 * the first sweeps, which time the tuning candidates). */
pulda_status pulda_batch_sweep(pulda_batch *b, int32_t n_sweeps);
pulda_status pulda_batch_sync(pulda_batch *b);
/* pulda_batch_get_z / pulda_batch_stats -- as pulda_get_z / pulda_stats for
 * chain `chain` (0-based); PULDA_ERR_INVALID if out of range. */
pulda_status pulda_batch_get_z(pulda_batch *b, int32_t chain, int16_t *z_host);
pulda_status pulda_batch_stats(pulda_batch *b, int32_t chain, pulda_sweep_stats *out);
/* pulda_batch_tuning -- the z-step warps per CTA and the cooperative
 * threshold in use (-1 = none), whether tuning is over, whether a sweep is
 * one persistent launch (1) or six launches (0), and the alias layout in use
 * (1 = threshold and topic arrays, 2 = packed slots; see pulda_options); any
 * pointer may be NULL. */
pulda_status pulda_batch_tuning(pulda_batch *b, int32_t *z_warps, int32_t *coop_min_len, int32_t *tuned,
                                int32_t *one_launch, int32_t *alias_layout);
/* pulda_barrier_selftest -- checks the grid barrier of the one-launch
 * batched sweep on the current device (the paper has no counterpart: this is
 * failure detection of the launch form).  `blocks` CTAs (at most one per SM,
 * so all resident) pass `rounds` barriers that expect blocks + missing
 * arrivals; *passed receives the barriers passed, summed over the CTAs.  With
 * missing = 0 every barrier opens: PULDA_OK, *passed = blocks * rounds.  With
 * missing > 0 none does: each CTA gives up after waiting 2 s and the call
 * returns PULDA_ERR_TIMEOUT, the device still usable.  Synchronous; allocates
 * 256 bytes.  Errors: PULDA_ERR_INVALID (sizes), PULDA_ERR_OOM, PULDA_ERR_CUDA. */
pulda_status pulda_barrier_selftest(int32_t blocks, int32_t missing, int32_t rounds, int32_t *passed);
/* pulda_batch_last_error -- as pulda_last_error; NULL = last failed pulda_batch_init. */
const char *pulda_batch_last_error(const pulda_batch *b);
void pulda_batch_free(pulda_batch *b);

/* ---------------------------------------------------------------- serving
 * A continuous-batching fold-in server on a handle's current Phi (Algorithm
 * 2's z-step with Phi held fixed, on documents that arrive over time).  A
 * worker thread admits waiting requests while a slot and a contiguous range
 * of the token arena are free (memory-based admission, first come first
 * served), advances every admitted request by up to `slice_tokens` tokens per
 * launch (one warp per request; one CTA of the cooperative z-step per request
 * of at least the handle's coop_min_len tokens -- 1,024 when it is 0, none
 * when -1 -- on a second stream while the active requests fill at most an
 * eighth of the resident warps; sweeps continuing within a launch) and
 * copies finished topics out.  A request's result equals pulda_infer on that
 * document alone with the same seed and n_sweeps: its random streams are keyed
 * by its own seed and token positions, never by its neighbours.
 * Do not run pulda_sweep / pulda_phi_step on the handle while a server is open
 * on it (Phi would change under the requests). */
typedef struct pulda_server pulda_server;

typedef struct {
    uint64_t req_id;
    int32_t status;      /* PULDA_OK, or PULDA_ERR_CUDA if a kernel reported an error */
    int32_t len;         /* tokens */
    int64_t submit_ns;   /* CLOCK_MONOTONIC at pulda_serve_submit */
    int64_t done_ns;     /* CLOCK_MONOTONIC when z_out had been written */
} pulda_result;

/* pulda_serve_open -- token_budget: tokens the arena holds (6 bytes each on
 * the device, 6 pinned on the host); max_slots: requests in flight;
 * slice_tokens: tokens a request
 * advances per launch, or 0 for launches of about 2 ms in which every request
 * advances as far as it gets (at least 32 tokens, in whole 32-token blocks,
 * while a 2 ms window from when a warp or CTA takes it up is open); results do
 * not depend on it.  Waits for the work queued on the handle's stream (the sweeps that
 * drew Phi) before the server's first launch.  Errors: PULDA_ERR_INVALID (no
 * Phi yet, token_budget or max_slots < 1, slice_tokens < 0),
 * PULDA_ERR_OOM, PULDA_ERR_CUDA, or a device error pulda_sync reports. */
pulda_status pulda_serve_open(pulda_handle *h, int64_t token_budget, int32_t max_slots, int64_t slice_tokens,
                              pulda_server **out);
/* pulda_serve_submit -- enqueue one document (thread safe).  words_host
 * int32[len] is copied; z_out_host int16[len] receives the topics and must stay
 * valid until the request is returned by pulda_serve_poll.  Errors:
 * PULDA_ERR_INVALID (len < 1 or beyond the arena, ids outside [0, V),
 * n_sweeps < 1, server closing), PULDA_ERR_BUSY (2^22 requests waiting),
 * PULDA_ERR_CUDA (the worker failed). */
pulda_status pulda_serve_submit(pulda_server *s, uint64_t req_id, uint64_t seed, const int32_t *words_host,
                                int32_t len, int32_t n_sweeps, int16_t *z_out_host);
/* pulda_serve_poll -- wait up to timeout_ms for finished requests and return
 * up to max_results of them (thread safe).  PULDA_ERR_TIMEOUT if none finished
 * in time; the wait is bounded, never indefinite. */
pulda_status pulda_serve_poll(pulda_server *s, pulda_result *out, int32_t max_results, int32_t *n_out,
                              int32_t timeout_ms);
/* pulda_serve_pending -- requests waiting for admission, requests in flight,
 * and launches so far (any pointer may be NULL). */
pulda_status pulda_serve_pending(pulda_server *s, int64_t *waiting, int64_t *running, int64_t *launches);
/* pulda_serve_stats -- out int64[8]: launches, requests completed, token
 * steps completed (tokens x sweeps), kernel nanoseconds, current slice,
 * largest number of requests in one launch, requests waiting, requests in
 * flight. */
pulda_status pulda_serve_stats(pulda_server *s, int64_t *out);
/* pulda_serve_close -- stop accepting, finish every submitted request, release
 * the server.  Returns the worker's error status, if any. */
pulda_status pulda_serve_close(pulda_server *s);

/* pulda_z_layout -- how the handle's corpus z-step is laid out (launch shape
 * only: results never depend on it): documents per warp of the main z-step
 * kernel (1 or 4), the number of (longest) documents resampled by one CTA
 * each, and, beside four per warp, the documents too long for it that run one
 * per warp (otherwise every document not on a CTA).  Any pointer may be NULL.
 * Errors: PULDA_ERR_INVALID (NULL handle). */
pulda_status pulda_z_layout(pulda_handle *h, int32_t *docs_per_warp, int64_t *coop_docs, int64_t *one_warp_docs);

/* pulda_stats -- counters of the most recent sweep (synchronises). */
pulda_status pulda_stats(pulda_handle *h, pulda_sweep_stats *out);

/* pulda_last_error -- human-readable description of the handle's last
 * failure, or ""; with h = NULL, the reason the calling thread's last
 * pulda_init failed. */
const char *pulda_last_error(const pulda_handle *h);

/* pulda_free -- release every resource of the handle (NULL is a no-op). */
void pulda_free(pulda_handle *h);

#ifdef __cplusplus
}
#endif
#endif
