// C ABI of the pulda sampler: argument validation, device buffers, and the
// order of kernel launches that makes one sweep (Algorithm 2, Section 3).
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pulda.h"
#include "handle.h"
#include "pulda_internal.h"

using namespace pulda;

namespace {

// An NVTX range over a scope (a no-op unless a profiler listens).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};


thread_local std::string g_init_error;

pulda_status fail(pulda_handle *h, pulda_status s, const char *fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return s;
}

#define CU(h, expr)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (expr);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail((h), e_ == cudaErrorMemoryAllocation ? PULDA_ERR_OOM : PULDA_ERR_CUDA,        \
                        "%s failed: %s", #expr, cudaGetErrorString(e_));                              \
    } while (0)

// inside pulda_init: record the failure and release the half-built handle
#define CUI(expr)                                                                                     \
    do {                                                                                              \
        cudaError_t e_ = (expr);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            pulda_status s_ = e_ == cudaErrorMemoryAllocation ? PULDA_ERR_OOM : PULDA_ERR_CUDA;       \
            fail(h, s_, "%s failed: %s", #expr, cudaGetErrorString(e_));                              \
            return bail(s_);                                                                          \
        }                                                                                             \
    } while (0)

template <typename T>
cudaError_t dalloc(pulda_handle *h, T **p, size_t count) {
    void *ptr = nullptr;
    cudaError_t e = dev_alloc(h->opt, h->stream, sizeof(T) * std::max<size_t>(count, 1), &ptr, false);
    if (e == cudaSuccess) h->allocs.push_back(ptr);
    *p = static_cast<T *>(ptr);
    return e;
}

// Smallest i in [0, n) with bad(i), else n, using up to 16 host threads.
template <typename F>
int64_t parallel_first(int64_t n, F bad) {
    const int64_t kChunk = int64_t(1) << 22;
    const int nt = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>({int64_t(16), (n + kChunk - 1) / kChunk,
                                                         static_cast<int64_t>(std::max(1u, std::thread::hardware_concurrency()))})));
    std::vector<int64_t> first(nt, n);
    auto scan = [&](int t) {
        const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
        for (int64_t i = lo; i < hi; ++i)
            if (bad(i)) { first[t] = i; return; }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(scan, t);
    scan(0);
    for (auto &x : th) x.join();
    return *std::min_element(first.begin(), first.end());
}

pulda_status check_corpus(pulda_handle *h, const int32_t *w, const int64_t *off, int64_t D, int V,
                          int64_t *N_out) {
    if (D < 0) return fail(h, PULDA_ERR_INVALID, "D must be >= 0 (got %lld)", (long long)D);
    if (D > 0 && !off) return fail(h, PULDA_ERR_INVALID, "doc_offsets is NULL");
    if (D > 0 && off[0] != 0) return fail(h, PULDA_ERR_INVALID, "doc_offsets[0] must be 0");
    for (int64_t d = 0; d < D; ++d) {
        if (off[d + 1] < off[d]) return fail(h, PULDA_ERR_INVALID, "doc_offsets decrease at document %lld", (long long)d);
        if (off[d + 1] - off[d] > (int64_t(1) << 22))
            return fail(h, PULDA_ERR_INVALID, "document %lld is longer than 2^22 tokens", (long long)d);
    }
    const int64_t N = D > 0 ? off[D] : 0;
    if (N >= (int64_t(1) << 31)) return fail(h, PULDA_ERR_INVALID, "corpus larger than 2^31-1 tokens");
    if (N > 0 && !w) return fail(h, PULDA_ERR_INVALID, "word_ids is NULL");
    // the first word id outside [0, V): chunks scanned by host threads, the
    // smallest bad position wins (the same answer as one scan)
    const int64_t bad = parallel_first(N, [&](int64_t i) { return w[i] < 0 || w[i] >= V; });
    if (bad < N)
        return fail(h, PULDA_ERR_INVALID, "word id %d at token %lld is outside [0, %d)", w[bad], (long long)bad, V);
    *N_out = N;
    return PULDA_OK;
}

// Topic histograms of the most frequent words, before the per-word pass.
cudaError_t run_heavy(pulda_handle *h) {
    if (h->n_heavy == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(h->heavy_hist, 0, sizeof(uint32_t) * static_cast<size_t>(h->n_heavy) * h->K, h->stream);
    if (e != cudaSuccess) return e;
    launch_heavy_hist(h->d_self, h->d_heavy_chunks, static_cast<int>(h->heavy_chunks.size()), h->K, h->stream);
    return cudaGetLastError();
}

// The per-sweep z-step counters start from zero at every z-step.
cudaError_t clear_z_counters(pulda_handle *h) {
    cudaError_t e = cudaMemsetAsync(h->stats + ST_TOKENS, 0, sizeof(unsigned long long) * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->stats + ST_SUMINT, 0, sizeof(unsigned long long) * 2, h->stream);
    return e;
}

// Documents in decreasing length (ties by index), so the persistent z-step
// starts the long ones first.
// Whether every document from position `from` of a length order (longest
// first) has at most kNarrowMaxLen tokens: the one-warp z-step over them can
// hold its counts in 16 bits.
bool narrow_from(const int64_t *off, const std::vector<int32_t> &order, int64_t from) {
    if (from >= static_cast<int64_t>(order.size())) return true;
    const int32_t d = order[static_cast<size_t>(from)];
    return off[d + 1] - off[d] <= kNarrowMaxLen;
}

std::vector<int32_t> length_order(const int64_t *off, int64_t D) {
    std::vector<int32_t> o(D);
    std::iota(o.begin(), o.end(), 0);
    std::stable_sort(o.begin(), o.end(), [&](int32_t a, int32_t b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    return o;
}

// Number of leading documents of a length-ordered schedule that the grouped
// z-step cannot take (longer than kMaxGroupDocLen tokens).
int64_t count_long(const int64_t *off, const std::vector<int32_t> &order) {
    int64_t n = 0;
    while (n < static_cast<int64_t>(order.size()) && off[order[n] + 1] - off[order[n]] > kMaxGroupDocLen) ++n;
    return n;
}

// Number of leading documents of a length-ordered schedule that the
// cooperative z-step takes: at least coop_min_len tokens (0 = automatic:
// longer than max(256, N / 8000), or N / 16000 beside the grouped z-step);
// none with coop_min_len < 0 or slices.
int64_t count_coop(const pulda_handle *h, const int64_t *off, const std::vector<int32_t> &order, int64_t N) {
    if (h->opt.coop_min_len < 0 || h->opt.slice_len > 0) return 0;
    const int64_t div = h->z_groups ? kCoopAutoDivGrouped : kCoopAutoDiv;
    const int64_t L = h->opt.coop_min_len > 0 ? h->opt.coop_min_len : std::max<int64_t>(kCoopAutoMin, N / div + 1);
    int64_t n = 0;
    while (n < static_cast<int64_t>(order.size()) && off[order[n] + 1] - off[order[n]] >= L) ++n;
    return n;
}

// One z-step over the documents doc_order[0..D) (longest first).  The
// first n_coop go to the cooperative kernel (a CTA each); with the grouped
// kernel, the documents after them that are too long for it (up to n_long)
// then run one per warp on the same stream, while the rest run four per warp
// (grouped) or one per warp on a second stream, joined back before the next
// step.
// `narrow`: every document the one-warp kernel gets (those after the first
// n_coop) has at most kNarrowMaxLen tokens.
pulda_status run_z(pulda_handle *h, const int64_t *doc_off, const int32_t *doc_order, int64_t D, int64_t n_long,
                   int64_t n_coop, const int32_t *w, int16_t *z, uint64_t seed, uint32_t sweep, int64_t index_base,
                   bool narrow) {
    CU(h, cudaMemsetAsync(h->work + 1, 0, 3 * sizeof(int), h->stream));
    ZArgs a = z_args(h, doc_off, doc_order, D, w, z, seed, sweep, index_base);
    a.narrow = narrow ? 1 : 0;
    const int64_t n_head = h->z_groups ? std::max(n_coop, n_long) : n_coop;
    auto launch_rest = [&](cudaStream_t st) {
        if (D <= n_head) return;
        ZArgs ar = a;
        ar.doc_order = doc_order + n_head;
        ar.D = D - n_head;
        if (h->z_groups) {
            ar.work = h->work + 2;
            launch_z_step_groups(ar, h->zg_grid, st);
        } else {
            launch_z_step(ar, h->z_warps, h->z_grid, st);
        }
    };
    if (n_head > 0) {
        CU(h, cudaEventRecord(h->ev_fork, h->stream));
        if (n_coop > 0) launch_z_step_coop(a, static_cast<int>(n_coop), h->work + 3, h->coop_grid, h->stream);
        if (n_head > n_coop) {
            ZArgs al = a;
            al.doc_order = doc_order + n_coop;
            al.D = n_head - n_coop;
            launch_z_step(al, h->z_warps, h->z_grid, h->stream);
        }
        CU(h, cudaStreamWaitEvent(h->stream2, h->ev_fork, 0));
        launch_rest(h->stream2);
        CU(h, cudaEventRecord(h->ev_join, h->stream2));
        CU(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    } else {
        launch_rest(h->stream);
    }
    CU(h, cudaGetLastError());
    return PULDA_OK;
}

}  // namespace

namespace pulda {
cudaError_t dev_alloc(const pulda_options &o, cudaStream_t st, size_t bytes, void **out, bool stream_ordered) {
    *out = nullptr;
    if (o.alloc) {
        void *p = o.alloc(bytes, st, o.alloc_ctx);
        if (!p) return cudaErrorMemoryAllocation;
        if (reinterpret_cast<uintptr_t>(p) & 255u) {
            o.free(p, st, o.alloc_ctx);
            return cudaErrorMisalignedAddress;
        }
        *out = p;
        return cudaSuccess;
    }
    return stream_ordered ? cudaMallocAsync(out, bytes, st) : cudaMalloc(out, bytes);
}

void dev_free(const pulda_options &o, cudaStream_t st, void *p, bool stream_ordered) {
    if (!p) return;
    if (o.alloc) o.free(p, st, o.alloc_ctx);
    else if (stream_ordered) cudaFreeAsync(p, st);
    else cudaFree(p);
}

PhiArgs phi_args(pulda_handle *h) {
    PhiArgs a{};
    a.K = h->K; a.V = h->V; a.seed = h->seed; a.sweep = static_cast<uint32_t>(h->sweep);
    a.perm = h->perm; a.word_off = h->word_off; a.word_order = h->word_order; a.z = h->z;
    a.tab = DevTables{h->t_thr, h->t_alias, h->t_off, h->t_lo, h->t_n, h->t_geo, h->t_gauss, static_cast<double>(h->beta)};
    a.nst_k = h->nst_k; a.nst_n = h->nst_n; a.nnz_n = h->nnz_n;
    a.cst_k = h->cst_k; a.cst_c = h->cst_c; a.nnz_c = h->nnz_c;
    a.S = h->S; a.rowbuf = h->rowbuf; a.col_ptr = h->col_ptr;
    a.topic = h->topic; a.c = h->c; a.q = h->q; a.athr = h->athr; a.atopic = h->atopic; a.apack = h->apack;
    a.A = h->A; a.vose_p = h->vose_p; a.vose_stack = h->vose_stack; a.bits = h->bits; a.KW = h->KW; a.KWp = h->KWp;
    a.qdense = h->qdense; a.dense_slot = h->dense_slot;
    a.alpha = h->alpha; a.work = h->work; a.stats = h->stats;
    a.heavy_row = h->heavy_row; a.heavy_hist = h->heavy_hist; a.n_heavy = h->n_heavy;
    a.gam = h->gam; a.Sd = h->Sd; a.invS = h->invS; a.invSf = h->invSf; a.dpart = h->dpart;
    return a;
}

ZArgs z_args(pulda_handle *h, const int64_t *doc_off, const int32_t *doc_order, int64_t D, const int32_t *w,
             int16_t *z, uint64_t seed, uint32_t sweep, int64_t index_base) {
    ZArgs a{};
    a.doc_off = doc_off; a.doc_order = doc_order; a.D = D; a.w = w; a.z = z;
    a.col_ptr = h->col_ptr; a.topic = h->topic; a.q = h->q; a.A = h->A; a.athr = h->athr; a.atopic = h->atopic;
    a.apack = h->apack;
    a.bits = h->bits; a.K = h->K; a.KW = h->KW; a.KWp = h->KWp; a.seed = seed; a.sweep = sweep; a.index_base = index_base;
    a.qdense = h->qdense; a.dense_slot = h->dense_slot;
    a.path = h->opt.zstep_path; a.work = h->work + 1; a.stats = h->stats;
    return a;
}


// Read-only view of a handle for other translation units of the library.
bool handle_view(pulda_handle *h, HandleView *out) {
    if (!h || !out) return false;
    out->stream = h->stream;
    out->device = h->device;
    out->K = h->K;
    out->V = h->V;
    out->have_phi = h->have_phi;
    out->z_warps = h->z_warps;
    out->z_grid = h->z_grid;
    out->zargs = z_args(h, nullptr, nullptr, 0, nullptr, nullptr, 0, 0, 0);
    return true;
}

int handle_fail(pulda_handle *h, int s, const char *msg) { return fail(h, static_cast<pulda_status>(s), "%s", msg); }
}  // namespace pulda

extern "C" {

pulda_status pulda_init(pulda_handle **out, const int32_t *word_ids, const int64_t *doc_offsets, int64_t D, int32_t K,
                        int32_t V, const float *alpha, float beta, uint64_t seed, const pulda_options *opt) {
    if (!out) return PULDA_ERR_INVALID;
    *out = nullptr;
    pulda_handle *h = new pulda_handle();
    // the handle is returned only on success: keep the reason of a failure
    // where pulda_last_error(NULL) finds it
    auto bail = [&](pulda_status s) { g_init_error = h->err; pulda_free(h); return s; };
    auto reject = bail;
    g_init_error.clear();
    if (K < 1 || K > kMaxK) { fail(h, PULDA_ERR_INVALID, "K must be in [1, %d] (got %d)", kMaxK, K); return reject(PULDA_ERR_INVALID); }
    if (V < 1) { fail(h, PULDA_ERR_INVALID, "V must be >= 1 (got %d)", V); return reject(PULDA_ERR_INVALID); }
    if (!(beta > 0.0f && beta <= 64.0f)) { fail(h, PULDA_ERR_INVALID, "beta must be in (0, 64]"); return reject(PULDA_ERR_INVALID); }
    if (!alpha) { fail(h, PULDA_ERR_INVALID, "alpha is NULL"); return reject(PULDA_ERR_INVALID); }
    for (int k = 0; k < K; ++k)
        if (!(alpha[k] > 0.0f && alpha[k] <= 256.0f)) {
            fail(h, PULDA_ERR_INVALID, "alpha[%d] must be in (0, 256]", k);
            return reject(PULDA_ERR_INVALID);
        }
    int64_t N = 0;
    if (check_corpus(h, word_ids, doc_offsets, D, V, &N) != PULDA_OK) return reject(PULDA_ERR_INVALID);
    if (opt) h->opt = *opt;
    if ((h->opt.alloc == nullptr) != (h->opt.free == nullptr)) {
        fail(h, PULDA_ERR_INVALID, "alloc and free must be set together");
        h->opt.alloc = nullptr;          // nothing was allocated: free nothing through it
        h->opt.free = nullptr;
        return reject(PULDA_ERR_INVALID);
    }
    if (h->opt.zstep_path < 0 || h->opt.zstep_path > 2) { fail(h, PULDA_ERR_INVALID, "zstep_path must be 0, 1 or 2"); return reject(PULDA_ERR_INVALID); }
    if (h->opt.phi_mode != 0 && h->opt.phi_mode != 1) {
        fail(h, PULDA_ERR_INVALID, "phi_mode must be 0 (Polya urn) or 1 (Dirichlet)");
        return reject(PULDA_ERR_INVALID);
    }
    if (h->opt.warps_per_block < 0 || h->opt.warps_per_block > kZWarps) {
        fail(h, PULDA_ERR_INVALID, "warps_per_block must be in [0, %d] (got %d)", kZWarps, h->opt.warps_per_block);
        return reject(PULDA_ERR_INVALID);
    }
    if (h->opt.docs_per_warp != 0 && h->opt.docs_per_warp != 1 && h->opt.docs_per_warp != 4) {
        fail(h, PULDA_ERR_INVALID, "docs_per_warp must be 0 (auto), 1 or 4");
        return reject(PULDA_ERR_INVALID);
    }
    if (h->opt.slice_len < 0 || (h->opt.slice_len > 0 && h->opt.docs_per_warp == 4)) {
        fail(h, PULDA_ERR_INVALID, "slice_len must be >= 0, and slices need docs_per_warp 0 or 1");
        return reject(PULDA_ERR_INVALID);
    }
    if (h->opt.alias_layout < 0 || h->opt.alias_layout > 2) {
        fail(h, PULDA_ERR_INVALID, "alias_layout must be 0 (default), 1 (threshold and topic arrays) or 2 (packed slots)");
        return reject(PULDA_ERR_INVALID);
    }
    if (h->opt.count_path != 0 && h->opt.count_path != 1) {
        fail(h, PULDA_ERR_INVALID, "count_path must be 0 (histogram) or 1 (sort)");
        return reject(PULDA_ERR_INVALID);
    }
    if (h->opt.count_path == 1 && static_cast<uint64_t>(K) * static_cast<uint64_t>(V) >= (uint64_t(1) << 32)) {
        fail(h, PULDA_ERR_INVALID, "count_path 1 needs V K < 2^32 (sort keys are 32-bit)");
        return reject(PULDA_ERR_INVALID);
    }
    if (h->opt.coop_min_len < -1) {
        fail(h, PULDA_ERR_INVALID, "coop_min_len must be -1 (never), 0 (auto) or a length");
        return reject(PULDA_ERR_INVALID);
    }
    if (h->opt.docs_per_warp == 4 && K > kMaxKGrouped) {
        fail(h, PULDA_ERR_INVALID, "docs_per_warp = 4 needs K <= 1024");
        return reject(PULDA_ERR_INVALID);
    }
    h->N = N; h->D = D; h->K = K; h->V = V; h->seed = seed; h->beta = beta;
    for (int k = 0; k < K; ++k) h->alpha_sum += static_cast<double>(alpha[k]);
    h->KW = (K + 31) / 32;
    h->KWp = bitmap_row_words(K);
    h->cap = static_cast<int64_t>(K) * V;
    cudaGetDevice(&h->device);
    if (h->opt.stream) {
        h->stream = static_cast<cudaStream_t>(h->opt.stream);
    } else {
        CUI(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    HostTables tab;
    if (build_host_tables(beta, &tab) != 0) { fail(h, PULDA_ERR_INVALID, "Poisson table construction failed"); return bail(PULDA_ERR_INVALID); }

#define ALLOC(ptr, n) do { cudaError_t e_ = dalloc(h, &(ptr), (n)); if (e_ != cudaSuccess) { \
        const pulda_status s_ = e_ == cudaErrorMemoryAllocation ? PULDA_ERR_OOM : PULDA_ERR_CUDA; \
        fail(h, s_, "allocation of %s (%zu entries) failed: %s", #ptr, (size_t)(n), cudaGetErrorString(e_)); \
        return bail(s_); } } while (0)
    ALLOC(h->w, N); ALLOC(h->doc_off, D + 1); ALLOC(h->z, N); ALLOC(h->doc_order, D);
    ALLOC(h->perm, N); ALLOC(h->word_off, V + 1); ALLOC(h->word_order, V); ALLOC(h->fill, V);
    ALLOC(h->alpha, K);
    ALLOC(h->t_thr, tab.thr.size()); ALLOC(h->t_alias, tab.alias.size()); ALLOC(h->t_off, kL + 1);
    ALLOC(h->t_lo, kL + 1); ALLOC(h->t_n, kL + 1); ALLOC(h->t_geo, kGeoLen); ALLOC(h->t_gauss, kGaussCells + 1);
    ALLOC(h->nst_k, N); ALLOC(h->nst_n, N); ALLOC(h->nnz_n, V);
    ALLOC(h->cst_k, h->cap); ALLOC(h->cst_c, h->cap); ALLOC(h->nnz_c, V);
    ALLOC(h->S, K); ALLOC(h->rowbuf, V); ALLOC(h->col_ptr, V + 1);
    ALLOC(h->topic, h->cap); ALLOC(h->c, h->cap); ALLOC(h->q, h->cap); ALLOC(h->athr, h->cap); ALLOC(h->atopic, h->cap);
    if (h->opt.alias_layout == 2) ALLOC(h->apack, h->cap);
    ALLOC(h->A, V); ALLOC(h->vose_p, h->cap); ALLOC(h->vose_stack, h->cap);
    if (K <= kMaxKBitmap) ALLOC(h->bits, static_cast<size_t>(V) * h->KWp);
    if (h->opt.phi_mode == 1) {
        ALLOC(h->gam, h->cap); ALLOC(h->Sd, K); ALLOC(h->invS, K); ALLOC(h->invSf, K);
        ALLOC(h->dpart, dir_part_count(V, K));
    }
    ALLOC(h->work, 4); ALLOC(h->stats, ST_TOTAL_SLOTS);
    if (h->opt.count_path == 1) ALLOC(h->sort_scratch, count_sort_scratch_words(N));
    cudaStream_t st = h->stream;
    CUI(cudaMemcpyAsync(h->w, word_ids, sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
    std::vector<int64_t> off0(1, 0);
    CUI(cudaMemcpyAsync(h->doc_off, D > 0 ? doc_offsets : off0.data(), sizeof(int64_t) * (D + 1), cudaMemcpyHostToDevice, st));
    std::vector<int32_t> dord = length_order(doc_offsets, D);
    CUI(cudaMemcpyAsync(h->doc_order, dord.data(), sizeof(int32_t) * D, cudaMemcpyHostToDevice, st));
    if (h->opt.slice_len > 0) {
        // documents longer than slice_len become slices {document, row, first token, tokens}
        const int64_t S = h->opt.slice_len;
        std::vector<int32_t> sdocs, shortd;
        std::vector<int4> items;
        for (int32_t d : dord) {
            const int64_t len = doc_offsets[d + 1] - doc_offsets[d];
            if (len > S) {
                const int row = static_cast<int>(sdocs.size());
                sdocs.push_back(d);
                for (int64_t a0 = 0; a0 < len; a0 += S)
                    items.push_back(make_int4(d, row, static_cast<int>(a0), static_cast<int>(std::min(S, len - a0))));
            } else {
                shortd.push_back(d);
            }
        }
        std::stable_sort(items.begin(), items.end(), [](const int4 &x, const int4 &y) { return x.w > y.w; });
        if (!sdocs.empty()) {
            ALLOC(h->sliced_docs, sdocs.size());
            ALLOC(h->slices, items.size());
            ALLOC(h->m0, sdocs.size() * static_cast<size_t>(K));
            CUI(cudaMemcpyAsync(h->sliced_docs, sdocs.data(), sizeof(int32_t) * sdocs.size(), cudaMemcpyHostToDevice, st));
            CUI(cudaMemcpyAsync(h->slices, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st));
            if (!shortd.empty()) {
                ALLOC(h->doc_order_short, shortd.size());
                CUI(cudaMemcpyAsync(h->doc_order_short, shortd.data(), sizeof(int32_t) * shortd.size(),
                                    cudaMemcpyHostToDevice, st));
            }
            CUI(cudaStreamSynchronize(st));
            h->n_sliced = static_cast<int>(sdocs.size());
            h->n_slices = static_cast<int>(items.size());
            h->D_short = static_cast<int64_t>(shortd.size());
        }
    }
    CUI(cudaMemcpyAsync(h->alpha, alpha, sizeof(float) * K, cudaMemcpyHostToDevice, st));
    CUI(cudaMemcpyAsync(h->t_thr, tab.thr.data(), sizeof(uint32_t) * tab.thr.size(), cudaMemcpyHostToDevice, st));
    CUI(cudaMemcpyAsync(h->t_alias, tab.alias.data(), sizeof(uint16_t) * tab.alias.size(), cudaMemcpyHostToDevice, st));
    CUI(cudaMemcpyAsync(h->t_off, tab.off.data(), sizeof(int32_t) * (kL + 1), cudaMemcpyHostToDevice, st));
    CUI(cudaMemcpyAsync(h->t_lo, tab.lo.data(), sizeof(int32_t) * (kL + 1), cudaMemcpyHostToDevice, st));
    CUI(cudaMemcpyAsync(h->t_n, tab.n.data(), sizeof(int32_t) * (kL + 1), cudaMemcpyHostToDevice, st));
    CUI(cudaMemcpyAsync(h->t_geo, tab.geo.data(), sizeof(uint32_t) * kGeoLen, cudaMemcpyHostToDevice, st));
    CUI(cudaMemcpyAsync(h->t_gauss, tab.gauss.data(), sizeof(double) * (kGaussCells + 1), cudaMemcpyHostToDevice, st));
    // word-major permutation and the word schedule (most tokens first)
    CUI(cudaGetLastError());            // nothing pending before the first launch
    launch_word_perm(N, V, h->w, h->word_off, h->fill, h->perm, st);
    CUI(cudaGetLastError());
    std::vector<int64_t> woff(V + 1);
    CUI(cudaMemcpyAsync(woff.data(), h->word_off, sizeof(int64_t) * (V + 1), cudaMemcpyDeviceToHost, st));
    CUI(cudaStreamSynchronize(st));
    std::vector<int32_t> word_order(V);
    std::iota(word_order.begin(), word_order.end(), 0);
    std::stable_sort(word_order.begin(), word_order.end(),
                     [&](int32_t a, int32_t b) { return woff[a + 1] - woff[a] > woff[b + 1] - woff[b]; });
    CUI(cudaMemcpyAsync(h->word_order, word_order.data(), sizeof(int32_t) * V, cudaMemcpyHostToDevice, st));
    // dense q rows for the most frequent words, within kDenseBytes
    if (K <= kMaxKBitmap && kDenseBytes > 0) {
        const int64_t cap = std::min<int64_t>(V, kDenseBytes / (static_cast<int64_t>(sizeof(uint32_t)) * K));
        std::vector<int32_t> slot(V, -1);
        int32_t n = 0;
        for (int32_t v : word_order) {   // every word, most frequent first, while the budget lasts
            if (n >= cap) break;
            slot[v] = n++;
        }
        if (n > 0) {
            ALLOC(h->dense_slot, V);
            // 32 words before the first row: the document side's empty gather
            // slots read the word before a lane's segment (times a zero count)
            ALLOC(h->qdense, static_cast<size_t>(n) * K + 32);
            CUI(cudaMemsetAsync(h->qdense, 0, 32 * sizeof(uint32_t), st));
            h->qdense += 32;
            CUI(cudaMemcpyAsync(h->dense_slot, slot.data(), sizeof(int32_t) * V, cudaMemcpyHostToDevice, st));
            CUI(cudaStreamSynchronize(st));
        }
        h->n_dense = n;
    }
    // the most frequent words are histogrammed in chunks by many CTAs
    {
        std::vector<int32_t> row(V, -1);
        for (int32_t v : word_order) {
            const int64_t cnt = woff[v + 1] - woff[v];
            if (cnt <= kHeavyWord) break;
            row[v] = h->n_heavy;
            for (int64_t b = woff[v]; b < woff[v + 1]; b += kHeavyChunk)
                h->heavy_chunks.push_back(HeavyChunk{0, h->n_heavy, v, 0, b, std::min(woff[v + 1], b + kHeavyChunk)});
            ++h->n_heavy;
        }
        ALLOC(h->heavy_row, V);
        ALLOC(h->d_self, 1);
        if (h->n_heavy > 0) {
            ALLOC(h->heavy_hist, static_cast<size_t>(h->n_heavy) * K);
            ALLOC(h->d_heavy_chunks, h->heavy_chunks.size());
            CUI(cudaMemcpyAsync(h->d_heavy_chunks, h->heavy_chunks.data(), sizeof(HeavyChunk) * h->heavy_chunks.size(),
                                cudaMemcpyHostToDevice, st));
        }
        CUI(cudaMemcpyAsync(h->heavy_row, row.data(), sizeof(int32_t) * V, cudaMemcpyHostToDevice, st));
        PhiArgs self = phi_args(h);
        CUI(cudaMemcpyAsync(h->d_self, &self, sizeof(PhiArgs), cudaMemcpyHostToDevice, st));
        CUI(cudaStreamSynchronize(st));
    }
#undef ALLOC
    CUI(cudaMemsetAsync(h->stats, 0, sizeof(unsigned long long) * ST_TOTAL_SLOTS, st));
    launch_init_z(N, K, seed, 0, h->z, st);
    CUI(cudaGetLastError());
    // launch shapes
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    int wpb = h->opt.warps_per_block;
    if (wpb <= 0) wpb = kZWarps;
    while (wpb > 1 && z_step_smem(K, wpb) > 160 * 1024) wpb >>= 1;
    h->z_warps = wpb;
    CUI(cudaGetLastError());
    // Four documents per warp share each token's fixed work (record, count
    // updates, scan, draw) over four tokens, but each lane then walks four
    // times the topics, so a token's intersection costs more and a document's
    // tokens advance about 3x slower.  Once the one-warp z-step spread small K
    // over 8 or 16 topics per lane it was faster at every K measured (z-step
    // ms, 100,000 documents of the large corpus: K = 50 10.2 vs 14.7 four per
    // warp, K = 100 10.4 vs 13.7, K = 200 10.3 vs 13.0), so auto takes one
    // per warp and four per warp is an explicit choice.  That needs every
    // word's dense q row; not with slices or the column-only path.
    const bool groups_ok = K <= kMaxKGrouped && h->n_dense == V && h->opt.slice_len == 0 && h->opt.zstep_path != 1;
    h->z_groups = groups_ok && h->opt.docs_per_warp == 4;
    h->n_long = count_long(doc_offsets, dord);
    h->n_coop = count_coop(h, doc_offsets, dord, N);
    h->narrow_z = narrow_from(doc_offsets, dord, h->n_coop);
    h->narrow_all = narrow_from(doc_offsets, dord, 0);
    // as many one-warp CTAs as fit with the corpus pass's count width (16-bit
    // counts halve the shared memory, which limits residency at large K); a
    // launch with 32-bit counts (a fold-in of long documents) queues the
    // CTAs that do not fit, each taking documents from the same counter
    h->z_grid = sms * z_step_blocks_per_sm(K, wpb, h->narrow_z);
    CUI(cudaGetLastError());
    h->coop_grid = sms * z_coop_blocks_per_sm(K);
    CUI(cudaGetLastError());
    CUI(cudaStreamCreateWithFlags(&h->stream2, cudaStreamNonBlocking));
    CUI(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CUI(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    if (h->z_groups) {
        h->zg_grid = sms * z_groups_blocks_per_sm(K);
        CUI(cudaGetLastError());
    }
    h->phi_grid = sms * phi_counts_blocks_per_sm(K);
    CUI(cudaGetLastError());
    CUI(cudaStreamSynchronize(st));
    *out = h;
    return PULDA_OK;
}

pulda_status pulda_phi_step(pulda_handle *h) {
    if (!h) return PULDA_ERR_INVALID;
    NvtxRange nv("pulda_phi_step");
    h->sweep += 1;
    cudaStream_t st = h->stream;
    CU(h, cudaMemsetAsync(h->stats, 0, sizeof(unsigned long long) * ST_COUNT, st));
    CU(h, cudaMemsetAsync(h->work, 0, sizeof(int), st));
    CU(h, cudaMemsetAsync(h->S, 0, sizeof(unsigned long long) * h->K, st));
    PhiArgs a = phi_args(h);
    if (h->opt.count_path == 1) {
        // n columns by sorting the tokens' (word, topic) keys
        launch_count_sort(h->w, h->z, h->N, h->K, h->V, h->word_off, h->nst_k, h->nst_n, h->nnz_n, h->sort_scratch,
                          h->stats, st);
        a.counted = 1;
    } else {
        CU(h, run_heavy(h));
    }
    if (h->gam) {
        // Algorithm 1: n columns, every Gamma draw, row sums, kept entries
        if (!a.counted) launch_phi_counts(a, false, h->phi_grid, st);
        launch_dir_phi(a, st);
    } else {
        // Algorithm 2: n columns with the Poisson draws, dead rows redrawn
        launch_phi_counts(a, true, h->phi_grid, st);
        launch_phi_fixup(a, st);
    }
    launch_colptr_scan(a, st);
    launch_phi_tables(a, st);
    CU(h, cudaGetLastError());
    h->have_phi = true;
    return PULDA_OK;
}

pulda_status pulda_z_step(pulda_handle *h) {
    if (!h) return PULDA_ERR_INVALID;
    NvtxRange nv("pulda_z_step");
    if (!h->have_phi) return fail(h, PULDA_ERR_INVALID, "no Phi drawn yet: call pulda_phi_step or pulda_sweep first");
    CU(h, clear_z_counters(h));
    if (h->n_slices > 0) {
        // long documents in stale-count slices: their pass-start counts, then
        // one launch over the slices and the other documents
        CU(h, cudaMemsetAsync(h->work + 1, 0, 2 * sizeof(int), h->stream));
        launch_slice_counts(h->doc_off, h->sliced_docs, h->n_sliced, h->z, h->K, h->m0, h->stream);
        ZArgs a = z_args(h, h->doc_off, h->doc_order_short, h->D_short, h->w, h->z, h->seed,
                         static_cast<uint32_t>(h->sweep), 0);
        a.slices = h->slices;
        a.n_slices = h->n_slices;
        a.m0 = h->m0;
        a.narrow = h->narrow_all ? 1 : 0;      // the slices start from whole documents' counts
        launch_z_step(a, h->z_warps, h->z_grid, h->stream);
        CU(h, cudaGetLastError());
        return PULDA_OK;
    }
    return run_z(h, h->doc_off, h->doc_order, h->D, h->n_long, h->n_coop, h->w, h->z, h->seed,
                 static_cast<uint32_t>(h->sweep), 0, h->narrow_z);
}

pulda_status pulda_sweep(pulda_handle *h, int32_t n_sweeps) {
    if (!h) return PULDA_ERR_INVALID;
    if (n_sweeps < 0) return fail(h, PULDA_ERR_INVALID, "n_sweeps must be >= 0");
    for (int32_t s = 0; s < n_sweeps; ++s) {
        pulda_status r = pulda_phi_step(h);
        if (r != PULDA_OK) return r;
        r = pulda_z_step(h);
        if (r != PULDA_OK) return r;
    }
    return PULDA_OK;
}

pulda_status pulda_sync_timeout(pulda_handle *h, int32_t timeout_ms) {
    if (!h) return PULDA_ERR_INVALID;
    if (timeout_ms < 0) return fail(h, PULDA_ERR_INVALID, "timeout_ms must be >= 0");
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        const cudaError_t q = cudaStreamQuery(h->stream);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) CU(h, q);
        if (std::chrono::steady_clock::now() >= t_end)
            return fail(h, PULDA_ERR_TIMEOUT, "the handle's work did not finish within %d ms", timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    return pulda_sync(h);
}

pulda_status pulda_sync(pulda_handle *h) {
    if (!h) return PULDA_ERR_INVALID;
    CU(h, cudaStreamSynchronize(h->stream));
    unsigned long long e = 0;
    CU(h, cudaMemcpy(&e, h->stats + ST_ERROR, sizeof e, cudaMemcpyDeviceToHost));
    if (e & ERR_DEGENERATE) return fail(h, PULDA_ERR_DEGENERATE, "a Phi row stayed all-zero after 2^20 redraws");
    if (e & ERR_INTERNAL) return fail(h, PULDA_ERR_CUDA, "z-step invariant violated (draw beyond the total mass)");
    if (e & ERR_GAMMA) return fail(h, PULDA_ERR_DEGENERATE, "a Gamma draw was rejected 2^16 times");
    if (e & ERR_BOUNDS) return fail(h, PULDA_ERR_CUDA, "an index read from device data was out of range (checked build)");
    if (e & ERR_BARRIER) return fail(h, PULDA_ERR_TIMEOUT, "a grid barrier of the one-launch batched sweep waited 2 s");
    return PULDA_OK;
}

pulda_status pulda_get_z(pulda_handle *h, int16_t *z_host) {
    if (!h || (!z_host && h->N)) return fail(h, PULDA_ERR_INVALID, "z_host is NULL");
    CU(h, cudaMemcpyAsync(z_host, h->z, sizeof(int16_t) * h->N, cudaMemcpyDeviceToHost, h->stream));
    return pulda_sync(h);
}

pulda_status pulda_get_z_dev(pulda_handle *h, int16_t *z_dev) {
    if (!h || (!z_dev && h->N)) return fail(h, PULDA_ERR_INVALID, "z_dev is NULL");
    CU(h, cudaMemcpyAsync(z_dev, h->z, sizeof(int16_t) * h->N, cudaMemcpyDeviceToDevice, h->stream));
    return PULDA_OK;
}

pulda_status pulda_set_z(pulda_handle *h, const int16_t *z_host, int64_t sweep) {
    if (!h) return PULDA_ERR_INVALID;
    if (sweep < 0 || sweep >= (int64_t(1) << 32)) return fail(h, PULDA_ERR_INVALID, "sweep out of range");
    for (int64_t i = 0; i < h->N; ++i)
        if (z_host[i] < 0 || z_host[i] >= h->K) return fail(h, PULDA_ERR_INVALID, "topic %d at token %lld out of range", z_host[i], (long long)i);
    CU(h, cudaMemcpyAsync(h->z, z_host, sizeof(int16_t) * h->N, cudaMemcpyHostToDevice, h->stream));
    h->sweep = sweep;
    h->have_phi = false;
    return pulda_sync(h);
}

pulda_status pulda_get_counts(pulda_handle *h, int32_t *n_kv, int32_t *m_dk) {
    if (!h) return PULDA_ERR_INVALID;
    cudaStream_t st = h->stream;
    if (n_kv) {
        // rebuild n from the current z (counts only, no draws)
        PhiArgs a = phi_args(h);
        CU(h, cudaMemsetAsync(h->work, 0, sizeof(int), st));
        CU(h, run_heavy(h));
        launch_phi_counts(a, false, h->phi_grid, st);
        int32_t *dn = nullptr;
        DevTemp tn(h->opt, st);
        CU(h, tn.get(&dn, static_cast<size_t>(h->K) * h->V));
        launch_n_dense(a, dn, st);
        CU(h, cudaMemcpyAsync(n_kv, dn, sizeof(int32_t) * static_cast<size_t>(h->K) * h->V, cudaMemcpyDeviceToHost, st));
    }
    if (m_dk && h->D > 0) {
        int32_t *dm = nullptr;
        DevTemp tm(h->opt, st);
        CU(h, tm.get(&dm, static_cast<size_t>(h->K) * h->D));
        launch_doc_topic(h->doc_off, h->D, h->z, h->K, dm, st);
        CU(h, cudaMemcpyAsync(m_dk, dm, sizeof(int32_t) * static_cast<size_t>(h->K) * h->D, cudaMemcpyDeviceToHost, st));
    }
    CU(h, cudaGetLastError());
    return pulda_sync(h);
}

pulda_status pulda_log_posterior(pulda_handle *h, double *out) {
    NvtxRange nv("pulda_log_posterior");
    if (!h) return PULDA_ERR_INVALID;
    if (!out) return fail(h, PULDA_ERR_INVALID, "out is NULL");
    cudaStream_t st = h->stream;
    // n from the current z (counts only, no draws), then the three reductions
    PhiArgs a = phi_args(h);
    CU(h, cudaMemsetAsync(h->work, 0, sizeof(int), st));
    CU(h, run_heavy(h));
    launch_phi_counts(a, false, h->phi_grid, st);
    unsigned char *scratch = nullptr;
    DevTemp ts(h->opt, st);
    CU(h, ts.get(&scratch, log_posterior_scratch_bytes(h->D, h->V, h->K)));
    launch_log_posterior(h->doc_off, h->D, h->z, h->K, h->alpha, h->alpha_sum, a, static_cast<double>(h->beta), scratch, st);
    CU(h, cudaGetLastError());
    CU(h, cudaMemcpyAsync(out, scratch, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    return pulda_sync(h);
}

pulda_status pulda_get_word_tables(pulda_handle *h, int64_t *col_ptr, int16_t *topic, uint32_t *c, int64_t *S,
                                   uint32_t *q, uint64_t *A, uint32_t *athr, int16_t *atopic, int64_t *nnz_inout) {
    if (!h || !nnz_inout) return fail(h, PULDA_ERR_INVALID, "nnz_inout is NULL");
    if (!h->have_phi) return fail(h, PULDA_ERR_INVALID, "no Phi drawn yet");
    cudaStream_t st = h->stream;
    int64_t nnz = 0;
    CU(h, cudaMemcpyAsync(&nnz, h->col_ptr + h->V, sizeof nnz, cudaMemcpyDeviceToHost, st));
    CU(h, cudaStreamSynchronize(st));
    const bool want = col_ptr || topic || c || q || athr || atopic;
    if (want && *nnz_inout < nnz) {
        int64_t have = *nnz_inout;
        *nnz_inout = nnz;
        return fail(h, PULDA_ERR_INVALID, "capacity %lld < nnz %lld", (long long)have, (long long)nnz);
    }
    *nnz_inout = nnz;
    if (col_ptr) CU(h, cudaMemcpyAsync(col_ptr, h->col_ptr, sizeof(int64_t) * (h->V + 1), cudaMemcpyDeviceToHost, st));
    if (topic) CU(h, cudaMemcpyAsync(topic, h->topic, sizeof(uint16_t) * nnz, cudaMemcpyDeviceToHost, st));
    if (c) CU(h, cudaMemcpyAsync(c, h->c, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToHost, st));
    if (S) CU(h, cudaMemcpyAsync(S, h->gam ? static_cast<const void *>(h->Sd) : static_cast<const void *>(h->S),
                                 sizeof(int64_t) * h->K, cudaMemcpyDeviceToHost, st));
    if (q) CU(h, cudaMemcpyAsync(q, h->q, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToHost, st));
    if (A) CU(h, cudaMemcpyAsync(A, h->A, sizeof(uint64_t) * h->V, cudaMemcpyDeviceToHost, st));
    if (athr) CU(h, cudaMemcpyAsync(athr, h->athr, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToHost, st));
    if (atopic) CU(h, cudaMemcpyAsync(atopic, h->atopic, sizeof(uint16_t) * nnz, cudaMemcpyDeviceToHost, st));
    return pulda_sync(h);
}

pulda_status pulda_get_phi(pulda_handle *h, int64_t *col_ptr, int16_t *topic, float *phi, int64_t *nnz_inout) {
    if (!h || !nnz_inout) return fail(h, PULDA_ERR_INVALID, "nnz_inout is NULL");
    if (!h->have_phi) return fail(h, PULDA_ERR_INVALID, "no Phi drawn yet");
    int64_t cap = *nnz_inout;
    pulda_status s = pulda_get_word_tables(h, col_ptr, topic, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nnz_inout);
    if (s != PULDA_OK) return s;
    if (phi) {
        const int64_t nnz = *nnz_inout;
        if (cap < nnz) return fail(h, PULDA_ERR_INVALID, "capacity %lld < nnz %lld", (long long)cap, (long long)nnz);
        cudaStream_t st = h->stream;
        float *dp = nullptr;
        DevTemp tp(h->opt, st);
        CU(h, tp.get(&dp, static_cast<size_t>(nnz)));
        PhiArgs a = phi_args(h);
        launch_phi_values(a, dp, st);
        CU(h, cudaMemcpyAsync(phi, dp, sizeof(float) * nnz, cudaMemcpyDeviceToHost, st));
        return pulda_sync(h);
    }
    return PULDA_OK;
}

pulda_status pulda_infer(pulda_handle *h, const int32_t *word_ids, const int64_t *doc_offsets, int64_t D_new,
                         int32_t n_sweeps, uint64_t seed, int16_t *z_out, int32_t *m_out) {
    NvtxRange nv("pulda_infer");
    if (!h) return PULDA_ERR_INVALID;
    if (!h->have_phi) return fail(h, PULDA_ERR_INVALID, "no Phi drawn yet: run a sweep before pulda_infer");
    if (n_sweeps < 0) return fail(h, PULDA_ERR_INVALID, "n_sweeps must be >= 0");
    int64_t N = 0;
    pulda_status s = check_corpus(h, word_ids, doc_offsets, D_new, h->V, &N);
    if (s != PULDA_OK) return s;
    if (D_new == 0) return PULDA_OK;
    cudaStream_t st = h->stream;
    int32_t *dw = nullptr, *dord = nullptr, *dm = nullptr;
    int64_t *doff = nullptr;
    int16_t *dz = nullptr;
    DevTemp tw(h->opt, st), toff(h->opt, st), tord(h->opt, st), tz(h->opt, st), tm(h->opt, st);
    CU(h, tw.get(&dw, static_cast<size_t>(N)));
    CU(h, toff.get(&doff, static_cast<size_t>(D_new + 1)));
    CU(h, tord.get(&dord, static_cast<size_t>(D_new)));
    CU(h, tz.get(&dz, static_cast<size_t>(N)));
    std::vector<int32_t> ord = length_order(doc_offsets, D_new);
    CU(h, cudaMemcpyAsync(dw, word_ids, sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
    CU(h, cudaMemcpyAsync(doff, doc_offsets, sizeof(int64_t) * (D_new + 1), cudaMemcpyHostToDevice, st));
    CU(h, cudaMemcpyAsync(dord, ord.data(), sizeof(int32_t) * D_new, cudaMemcpyHostToDevice, st));
    launch_init_z(N, h->K, seed, 0, dz, st);
    CU(h, clear_z_counters(h));
    const int64_t n_long = count_long(doc_offsets, ord);
    const int64_t n_coop = count_coop(h, doc_offsets, ord, N);
    const bool narrow = narrow_from(doc_offsets, ord, n_coop);
    for (int32_t sw = 1; sw <= n_sweeps; ++sw) {
        s = run_z(h, doff, dord, D_new, n_long, n_coop, dw, dz, seed, static_cast<uint32_t>(sw), 0, narrow);
        if (s != PULDA_OK) return s;
    }
    if (z_out) CU(h, cudaMemcpyAsync(z_out, dz, sizeof(int16_t) * N, cudaMemcpyDeviceToHost, st));
    if (m_out) {
        CU(h, tm.get(&dm, static_cast<size_t>(D_new) * h->K));
        launch_doc_topic(doff, D_new, dz, h->K, dm, st);
        CU(h, cudaMemcpyAsync(m_out, dm, sizeof(int32_t) * static_cast<size_t>(D_new) * h->K, cudaMemcpyDeviceToHost, st));
    }
    CU(h, cudaGetLastError());
    return pulda_sync(h);
}

pulda_status pulda_z_layout(pulda_handle *h, int32_t *docs_per_warp, int64_t *coop_docs, int64_t *one_warp_docs) {
    if (!h) return PULDA_ERR_INVALID;
    if (docs_per_warp) *docs_per_warp = h->z_groups ? 4 : 1;
    if (coop_docs) *coop_docs = h->n_coop;
    if (one_warp_docs) {
        const int64_t head = h->z_groups ? std::max(h->n_coop, h->n_long) : h->n_coop;
        *one_warp_docs = h->z_groups ? head - h->n_coop : h->D - h->n_coop;
    }
    return PULDA_OK;
}

pulda_status pulda_stats(pulda_handle *h, pulda_sweep_stats *out) {
    if (!h || !out) return PULDA_ERR_INVALID;
    pulda_status s = pulda_sync(h);
    if (s != PULDA_OK) return s;
    unsigned long long st[ST_TOTAL_SLOTS];
    CU(h, cudaMemcpy(st, h->stats, sizeof st, cudaMemcpyDeviceToHost));
    out->tokens = static_cast<int64_t>(st[ST_TOKENS]);
    out->a_branch = static_cast<int64_t>(st[ST_ABRANCH]);
    out->sum_min = static_cast<int64_t>(st[ST_SUMMIN]);
    out->zero_mass = static_cast<int64_t>(st[ST_ZEROMASS]);
    out->dead_rows = static_cast<int64_t>(st[ST_DEADROWS]);
    out->nnz_phi = static_cast<int64_t>(st[ST_NNZPHI]);
    out->sweep = h->sweep;
    out->cum_tokens = static_cast<int64_t>(st[ST_COUNT + ST_TOKENS]);
    out->cum_a_branch = static_cast<int64_t>(st[ST_COUNT + ST_ABRANCH]);
    out->cum_sum_min = static_cast<int64_t>(st[ST_COUNT + ST_SUMMIN]);
    out->cum_zero_mass = static_cast<int64_t>(st[ST_COUNT + ST_ZEROMASS]);
    out->sum_inter = static_cast<int64_t>(st[ST_SUMINT]);
    out->docside = static_cast<int64_t>(st[ST_DOCSIDE]);
    out->cum_sum_inter = static_cast<int64_t>(st[ST_COUNT + ST_SUMINT]);
    out->cum_docside = static_cast<int64_t>(st[ST_COUNT + ST_DOCSIDE]);
    return PULDA_OK;
}

const char *pulda_last_error(const pulda_handle *h) { return h ? h->err.c_str() : g_init_error.c_str(); }

void pulda_free(pulda_handle *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void *p : h->allocs) dev_free(h->opt, h->stream, p, false);
    if (h->stream2) {
        cudaStreamSynchronize(h->stream2);
        cudaStreamDestroy(h->stream2);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
