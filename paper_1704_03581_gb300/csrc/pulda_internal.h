// Internal declarations of the pulda CUDA library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace pulda {

// Alias tables are built for Poisson rates beta + l with l <= kL; larger
// counts use a rounded Gaussian ("Efficient sampling of Phi", L = 100).
constexpr int kL = 100;
// Length of the geometric-gap CDF table used to skip over entries whose
// Poisson rate is beta alone.
constexpr int kGeoLen = 1024;
// Equiprobable cells of the inverse-normal table.
constexpr int kGaussCells = 65536;
// The alpha part of the z conditional is held in units of 2^-16 q.
constexpr int kFracBits = 16;
// Dead-row redraw attempts before giving up.
constexpr uint32_t kMaxRedraw = 1u << 20;
// Largest K the kernels' shared-memory layouts accept.
constexpr int kMaxK = 16384;
// The bitmap intersection path of the z-step: the one-warp kernel's lane
// holds up to two 32-topic words (64 topics), the cooperative kernel's slot
// part of one.
constexpr int kMaxKBitmap = 2048;
// Four documents per warp: each of a document's 8 lanes holds up to four
// words.
constexpr int kMaxKGrouped = 1024;
// Words of a word's bitmap row: ceil(K / 32) rounded up to 8 times a power
// of two, so each of the grouped z-step's 8 lanes per document reads 1, 2 or
// 4 consecutive words with one aligned load (the words past ceil(K / 32) are
// zero); 64 above 1024 topics.
__host__ __device__ inline int bitmap_row_words(int K) {
    const int per_lane = (((K + 31) / 32) + 7) / 8;
    return 8 * (per_lane <= 1 ? 1 : per_lane <= 2 ? 2 : per_lane <= 4 ? 4 : 8);
}
// Warps per CTA of the warp-per-document z-step: the default and the largest
// accepted (the kernel's launch bounds are sized for it).
#ifndef PULDA_ZWARPS
#define PULDA_ZWARPS 4
#endif
constexpr int kZWarps = PULDA_ZWARPS;
// The batched (many-chain) z-step: the largest CTA in warps (its tuning
// candidates are the powers of two up to it) and the CTAs per SM its launch
// bounds ask for.
#ifndef PULDA_MULTI_WARPS
#define PULDA_MULTI_WARPS 8
#endif
#ifndef PULDA_MULTI_MINB
#define PULDA_MULTI_MINB 3
#endif
constexpr int kMultiWarps = PULDA_MULTI_WARPS;
// Words with tokens, most frequent first, also keep their fixed-point
// weights q as dense K-entry rows, up to this many bytes (K <= kMaxKBitmap):
// the z-step's document side reads q at topic k there.  A word without a row
// is always iterated on its column side (the same sums).
#ifndef PULDA_DENSE_BYTES
#define PULDA_DENSE_BYTES (2048ll << 20)
#endif
constexpr long long kDenseBytes = PULDA_DENSE_BYTES;

// Philox stream tags (counter word 3 = tag << 28 | aux).
enum : uint32_t { TAG_INIT = 1, TAG_POIS = 2, TAG_BETA = 3, TAG_REDRAW_POIS = 4, TAG_REDRAW_BETA = 5, TAG_Z = 6,
                  TAG_GAMMA = 7, TAG_GAMMA_BOOST = 8 };
// Dirichlet Phi-step (Algorithm 1): rows are summed in chunks of this many
// words, and a Gamma draw gives up after this many rejected attempts.
constexpr int kDirChunk = 256;
constexpr uint32_t kMaxGammaTry = 1u << 16;

// Slots of the per-sweep counter block on the device.
enum : int { ST_TOKENS = 0, ST_ABRANCH, ST_SUMMIN, ST_ZEROMASS, ST_DEADROWS, ST_NNZPHI, ST_ERROR, ST_SUMINT,
             ST_DOCSIDE, ST_COUNT = 12 };
// Running totals of the z-step slots live at ST_COUNT + slot and are cleared
// only at pulda_init.
constexpr int ST_TOTAL_SLOTS = 2 * ST_COUNT;
enum : unsigned long long { ERR_DEGENERATE = 1, ERR_INTERNAL = 2, ERR_GAMMA = 4, ERR_BOUNDS = 8, ERR_BARRIER = 16 };

// Fixed tables of one beta, built on the host once.
struct HostTables {
    std::vector<uint32_t> thr;     // alias thresholds of every table, concatenated
    std::vector<uint16_t> alias;   // alias outcome, as an offset from the table's lo
    std::vector<int32_t> off;      // [kL+1] start of table t (t = 0: zero-truncated Pois(beta); t = l: Pois(beta+l))
    std::vector<int32_t> lo;       // [kL+1] smallest value of table t
    std::vector<int32_t> n;        // [kL+1] support size of table t
    std::vector<uint32_t> geo;     // [kGeoLen] P(gap <= g) * 2^32
    std::vector<double> gauss;     // [kGaussCells+1] inverse-normal nodes
};
int build_host_tables(float beta, HostTables *out);

// Device view of the same tables.
struct DevTables {
    const uint32_t *thr;
    const uint16_t *alias;
    const int32_t *off;
    const int32_t *lo;
    const int32_t *n;
    const uint32_t *geo;
    const double *gauss;
    double beta;
};

// Everything the Phi-step kernels read and write.
struct PhiArgs {
    int K, V;
    uint64_t seed;
    uint32_t sweep;
    const uint32_t *sweep_ptr;  // if set, the sweep counter is read here (graph replay)
    const int32_t *perm;        // [N] token ids grouped by word
    const int64_t *word_off;    // [V+1]
    const int32_t *word_order;  // [V] words by decreasing token count
    const int16_t *z;           // [N]
    DevTables tab;
    // staging: n columns at word_off, c columns at v*K (capacity K each)
    uint16_t *nst_k; uint32_t *nst_n; int32_t *nnz_n;
    uint16_t *cst_k; uint32_t *cst_c; int32_t *nnz_c;
    unsigned long long *S;      // [K] row sums S_k
    uint32_t *rowbuf;           // [V] scratch of the dead-row redraw
    int64_t *col_ptr;           // [V+1]
    // final per-word tables, at col_ptr
    uint16_t *topic; uint32_t *c; uint32_t *q; uint32_t *athr; uint16_t *atopic;
    // the alias slots packed as {threshold, column topic | alias topic << 16}
    // (written beside athr / atopic when set; the z-step then reads one 8-byte
    // slot per alias draw instead of a threshold and a topic)
    uint2 *apack;
    unsigned long long *A;      // [V]
    unsigned long long *vose_p; // [cap] scratch
    uint16_t *vose_stack;       // [cap] scratch
    uint32_t *bits;             // [V * KWp] nonzero-topic bits of each word's column, or null
    int KW, KWp;
    uint32_t *qdense;           // [n_dense * K] q by topic (0 off the column) or null
    const int32_t *dense_slot;  // [V] row of the word in qdense, or -1
    const float *alpha;         // [K]
    int *work;                  // dynamic word counter
    unsigned long long *stats;  // [ST_COUNT]
    // words with more than kHeavyWord tokens get their topic histogram from a
    // separate pass split over many CTAs
    const int32_t *heavy_row;   // [V] row of the word in heavy_hist, or -1
    uint32_t *heavy_hist;       // [n_heavy * K]
    int n_heavy;
    // Dirichlet Phi (Algorithm 1); gam is null for the Polya urn
    float *gam;                 // [V * K] Gamma draws, word-major
    double *Sd;                 // [K] row sums
    double *invS;               // [K] 1 / S_k (0 for an all-zero row)
    float *invSf;               // [K] 1 / S_k rounded to float (screening only)
    double *dpart;              // [ceil(V / kDirChunk) * K] chunk sums of the rows
    int counted;                // the n columns are already built (sort path): read them, do not histogram
};

// A word with more tokens than this is histogrammed in chunks of kHeavyChunk
// tokens by several CTAs before the per-word Phi-step pass.
constexpr int64_t kHeavyWord = int64_t(1) << 17;
constexpr int64_t kHeavyChunk = int64_t(1) << 16;
// One chunk of a heavy word: chain, row in heavy_hist, word, token range.
struct HeavyChunk {
    int32_t chain, row, v, pad;
    int64_t begin, end;
};
void launch_heavy_hist(const PhiArgs *chains, const HeavyChunk *chunks, int n_chunks, int kmax, cudaStream_t st);
void launch_phi_tables_multi(const PhiArgs *chains, const int2 *items, int n_items, cudaStream_t st);

struct ZArgs {
    const int64_t *doc_off;     // [D+1]
    const int32_t *doc_order;   // [D] documents by decreasing length
    int64_t D;
    const int32_t *w;           // [N]
    int16_t *z;                 // [N]
    const int64_t *col_ptr;
    const uint16_t *topic;
    const uint32_t *q;
    const unsigned long long *A;
    const uint32_t *athr;
    const uint16_t *atopic;
    const uint2 *apack;         // packed alias slots (PhiArgs::apack) or null: read athr / topic / atopic
    const uint32_t *bits;       // [V * KWp] nonzero-topic bits of each word's column; null when K > kMaxKBitmap
    const uint32_t *qdense;     // dense q rows of the most frequent words, or null
    const int32_t *dense_slot;  // [V] row in qdense or -1
    // stale-count slices of long documents (k_z_step only): {row in m0, the
    // document, first token, tokens} is {y, x, z, w}; taken before the D documents
    const int4 *slices;
    int n_slices;
    const uint32_t *m0;         // [rows * K] pass-start counts of the sliced documents
    int K, KW, KWp;
    uint64_t seed;
    uint32_t sweep;
    const uint32_t *sweep_ptr;  // if set, the sweep counter is read here (graph replay)
    int64_t index_base;         // RNG index of token 0
    int path;                   // 0 auto, 1 column, 2 document topics
    int narrow;                 // 1: every document of the launch has fewer than 2^16 tokens (16-bit counts)
    int *work;
    unsigned long long *stats;
};

// Launchers (kernels.cu).  All are asynchronous on `st`.
void launch_init_z(int64_t N, int K, uint64_t seed, int64_t index_base, int16_t *z, cudaStream_t st);
void launch_word_perm(int64_t N, int V, const int32_t *w, int64_t *word_off, int32_t *fill, int32_t *perm,
                      cudaStream_t st);
void launch_phi_counts(const PhiArgs &a, bool draw, int grid, cudaStream_t st);
void launch_phi_fixup(const PhiArgs &a, cudaStream_t st);
void launch_colptr_scan(const PhiArgs &a, cudaStream_t st);
void launch_phi_tables(const PhiArgs &a, cudaStream_t st);
void launch_z_step(const ZArgs &a, int warps_per_block, int grid, cudaStream_t st);
// The longest documents, doc_order[0 .. n_coop), one CTA of four warps each;
// `work` is a counter zeroed before the launch.
void launch_z_step_coop(const ZArgs &a, int n_coop, int *work, int grid, cudaStream_t st);
int z_coop_blocks_per_sm(int K);
// Automatic threshold of the cooperative z-step: a document on one warp that
// shares its SM with the rest of the pass takes about 3.3 us per token while
// the pass streams ~2.4 G tokens/s, so one longer than N / 8000 tokens would
// outlast the pass.
constexpr int64_t kCoopAutoDiv = 8000;
constexpr int64_t kCoopAutoMin = 256;
// The same beside the grouped z-step, whose pass is faster and whose
// documents each advance more slowly (four share a warp's issue slots).
#ifndef PULDA_COOP_DIV_GROUPED
#define PULDA_COOP_DIV_GROUPED 16000
#endif
constexpr int64_t kCoopAutoDivGrouped = PULDA_COOP_DIV_GROUPED;
// Pass-start topic counts of the documents that the z-step takes in slices.
void launch_slice_counts(const int64_t *doc_off, const int32_t *sliced_docs, int n, const int16_t *z, int K,
                         uint32_t *m0, cudaStream_t st);
size_t z_step_smem(int K, int warps_per_block, bool narrow = false);
size_t phi_counts_smem(int K);
void launch_doc_topic(const int64_t *doc_off, int64_t D, const int16_t *z, int K, int32_t *m_dk, cudaStream_t st);
void launch_n_dense(const PhiArgs &a, int32_t *n_kv, cudaStream_t st);
void launch_phi_values(const PhiArgs &a, float *phi, cudaStream_t st);
int z_step_blocks_per_sm(int K, int warps_per_block, bool narrow = false);
// Grouped z-step (zgroup.cu): 4 documents per warp, 8 lanes each, K <=
// kMaxKGrouped, documents of at most kMaxGroupDocLen tokens, every word with a
// dense q row; the warps of a CTA are z_groups_warps().
constexpr int kMaxGroupDocLen = 65535;
// A one-warp z-step launch whose documents have at most this many tokens each
// keeps m_d's counts in 16 bits (ZArgs::narrow).
constexpr int64_t kNarrowMaxLen = 65535;
void launch_z_step_groups(const ZArgs &a, int grid, cudaStream_t st);
int z_groups_blocks_per_sm(int K);
int phi_counts_blocks_per_sm(int K);

// The count rebuild by sorting (countsort.cu): every token's key w K + z
// radix-sorted, runs of equal keys -> the n columns (nst_k, nst_n at
// word_off, nnz_n), bit-identical to the histogram pass's.  Needs V K < 2^32
// and count_sort_scratch_words(N) words of scratch.
size_t count_sort_scratch_words(int64_t N);
void launch_count_sort(const int32_t *w, const int16_t *z, int64_t N, int K, int V, const int64_t *word_off,
                       uint16_t *nst_k, uint32_t *nst_n, int32_t *nnz_n, uint32_t *scratch,
                       unsigned long long *stats, cudaStream_t st);

// Dirichlet Phi-step (dirichlet.cu), after the count-only pass has built the
// n columns: Gamma draws, row sums, and the kept entries staged in cst_k /
// cst_c (the draws' float bits) with nnz_c; the column scan and the table
// kernel follow as for the Polya urn.
void launch_dir_phi(const PhiArgs &a, cudaStream_t st);
size_t dir_part_count(int V, int K);

// Log-posterior diagnostic (diag.cu).  `counts` holds the n columns rebuilt
// from the current z (the count-only Phi-step pass); `scratch` is device
// memory of log_posterior_scratch_bytes(D, V, K) bytes whose first three
// doubles receive {total, document sum, topic sum}.
size_t log_posterior_scratch_bytes(int64_t D, int V, int K);
void launch_log_posterior(const int64_t *doc_off, int64_t D, const int16_t *z, int K, const float *alpha, double asum,
                          const PhiArgs &counts, double beta, void *scratch, cudaStream_t st);

// The grid barrier of the one-launch batched sweep (device memory, zeroed).
struct GridBarrier {
    unsigned count;
    unsigned gen;
};

// One sweep of many chains: six launches, every kernel over all chains'
// work items, or one persistent launch doing the same.  Pointers are device
// memory.
struct BatchLaunch {
    const HeavyChunk *heavy;     // heavy-word histogram chunks of every chain
    int n_heavy;
    const PhiArgs *phi;          // [n_chains], sweep_ptr = sweep
    const ZArgs *z;              // [n_chains], sweep_ptr = sweep
    int n_chains;
    const int2 *phi_items;       // (chain, word), most tokens first
    int n_phi_items;
    const int2 *z_items;         // (chain, document), longest first
    int n_z_items;
    uint32_t *sweep;             // shared sweep counter, advanced by the first launch
    int *work;                   // [4] dynamic work queues
    int kmax;                    // largest K of the chains
    int narrow;                  // 1: every document of every chain has fewer than 2^16 tokens
    int phi_grid, z_grid, z_warps;
    // the first n_coop z_items go to the cooperative z-step on `st`, the rest
    // to the one-warp kernel on stream2 (forked and joined with the events)
    int n_coop, coop_grid;
    cudaStream_t stream2;
    cudaEvent_t ev_fork, ev_join;
    // the one-launch form: its grid (all CTAs resident) and barrier
    int persist_grid;
    GridBarrier *bar;
};
void launch_batch_sweep(const BatchLaunch &b, cudaStream_t st);
// The same sweep as one cooperative launch (no cooperative z-step: every
// document one per warp); needs persist_grid <= SMs x
// batch_persistent_blocks_per_sm(kmax).
cudaError_t launch_batch_sweep_persistent(const BatchLaunch &b, cudaStream_t st);
int batch_persistent_blocks_per_sm(int kmax, bool narrow);
// The grid barrier's self-test: `blocks` resident CTAs pass `rounds`
// barriers that expect blocks + missing arrivals.
cudaError_t launch_barrier_selftest(GridBarrier *bar, int blocks, int missing, int rounds, unsigned long long *err,
                                    unsigned *passed, cudaStream_t st);
int batch_phi_blocks_per_sm(int kmax);
int batch_z_blocks_per_sm(int kmax, int warps, bool narrow);
int batch_coop_blocks_per_sm(int kmax);
size_t z_coop_multi_smem(int kmax);
// The cooperative z-step over (chain, document) items (coop.cu).
void launch_z_step_coop_multi(const ZArgs *chains, const int2 *items, int n_items, int *work, int kmax, int grid,
                              cudaStream_t st);

// A request being folded in by the server (device slot table entry).
struct ServeSlot {
    int64_t off;          // first token in the arena
    int32_t len;          // tokens (>= 1)
    int32_t pos;          // next position of the current pass
    uint32_t sweep;       // current pass; 0 = initial topics not drawn yet
    uint32_t sweep_end;   // 1 + sweeps requested: done when sweep reaches it
    uint64_t seed;        // the request's Philox key
};
// Each active slot advances by up to `slice` tokens, one warp per slot; with
// window_ns > 0 also stopping at the first 32-token block boundary window_ns
// after the launch starts (every slot does at least one block).
// `narrow`: every active request of the launch has at most kNarrowMaxLen tokens.
void launch_serve_step(const ZArgs &a, ServeSlot *slots, const int32_t *active, int n_active, const int32_t *arena_w,
                       int16_t *arena_z, int64_t slice, int *work, int warps_per_block, int grid, uint64_t window_ns,
                       bool narrow, cudaStream_t st);
int serve_blocks_per_sm(int K, int warps_per_block);
// The same with one CTA (the cooperative z-step) per slot, for long requests.
void launch_serve_step_coop(const ZArgs &a, ServeSlot *slots, const int32_t *active, int n_active,
                            const int32_t *arena_w, int16_t *arena_z, int64_t slice, int *work, int grid,
                            uint64_t window_ns, cudaStream_t st);
int serve_coop_blocks_per_sm(int K);
// Requests at least this long are served by the cooperative kernel when the
// handle's coop_min_len is 0 (automatic).
constexpr int64_t kServeCoopAuto = 1024;

// What another translation unit needs to launch the z-step on a handle's
// current Phi (api.cpp).
struct HandleView {
    cudaStream_t stream;
    int device;      // the device the handle was created on
    int K, V;
    bool have_phi;
    int z_warps, z_grid;
    ZArgs zargs;     // Phi tables, K, path; corpus, RNG and scratch fields unset
};
}  // namespace pulda
struct pulda_handle;
namespace pulda {
bool handle_view(pulda_handle *h, HandleView *out);
int handle_fail(pulda_handle *h, int status, const char *msg);

}  // namespace pulda
