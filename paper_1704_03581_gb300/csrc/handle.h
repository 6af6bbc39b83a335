// The state behind a pulda_handle (internal to the library).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pulda.h"
#include "pulda_internal.h"

struct pulda_handle {
    std::string err;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    pulda_options opt{};
    int device = 0;
    int64_t N = 0, D = 0;
    int K = 0, V = 0, KW = 0, KWp = 0;
    uint64_t seed = 0;
    int64_t sweep = 0;
    bool have_phi = false;
    float beta = 0;
    double alpha_sum = 0;       // sum_k alpha_k in double, index order
    int z_warps = 8, z_grid = 0, phi_grid = 0;
    bool z_groups = false;      // grouped z-step (four documents per warp) in use
    int zg_grid = 0;
    int64_t n_long = 0;         // documents too long for the grouped z-step (first in doc_order)
    int64_t n_coop = 0;         // documents the cooperative z-step takes (first in doc_order)
    bool narrow_z = false;      // the one-warp z-step's documents (after n_coop) fit 16-bit counts
    bool narrow_all = false;    // every document does
    int coop_grid = 0;
    cudaStream_t stream2 = nullptr;                       // the one-warp z-step beside the cooperative one
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<void *> allocs;
    // corpus and state
    int32_t *w = nullptr; int64_t *doc_off = nullptr; int16_t *z = nullptr; int32_t *doc_order = nullptr;
    int32_t *perm = nullptr; int64_t *word_off = nullptr; int32_t *word_order = nullptr; int32_t *fill = nullptr;
    float *alpha = nullptr;
    // fixed tables
    uint32_t *t_thr = nullptr; uint16_t *t_alias = nullptr; int32_t *t_off = nullptr, *t_lo = nullptr, *t_n = nullptr;
    uint32_t *t_geo = nullptr; double *t_gauss = nullptr;
    // Phi-step buffers
    uint16_t *nst_k = nullptr; uint32_t *nst_n = nullptr; int32_t *nnz_n = nullptr;
    uint16_t *cst_k = nullptr; uint32_t *cst_c = nullptr; int32_t *nnz_c = nullptr;
    unsigned long long *S = nullptr; uint32_t *rowbuf = nullptr; int64_t *col_ptr = nullptr;
    // stale-count slices (slice_len > 0): the documents longer than it, their
    // slices, their pass-start counts, and the order of the other documents
    int32_t *sliced_docs = nullptr; int n_sliced = 0;
    int4 *slices = nullptr; int n_slices = 0;
    uint32_t *m0 = nullptr;
    int32_t *doc_order_short = nullptr; int64_t D_short = 0;
    // dense q rows of the most frequent words (z-step document side)
    uint32_t *qdense = nullptr; int32_t *dense_slot = nullptr; int n_dense = 0;
    // Dirichlet Phi (Algorithm 1), allocated in that mode only
    float *gam = nullptr, *invSf = nullptr; double *Sd = nullptr, *invS = nullptr, *dpart = nullptr;
    uint16_t *topic = nullptr; uint32_t *c = nullptr, *q = nullptr, *athr = nullptr; uint16_t *atopic = nullptr;
    uint2 *apack = nullptr;     // packed alias slots (alias_layout 2), else null
    unsigned long long *A = nullptr, *vose_p = nullptr; uint16_t *vose_stack = nullptr; uint32_t *bits = nullptr;
    int *work = nullptr;
    unsigned long long *stats = nullptr;
    uint32_t *sort_scratch = nullptr;   // count_path 1: keys, run ids, scan sums
    int64_t cap = 0;   // capacity of the per-word tables: K * V entries
    // words histogrammed by several CTAs (more than kHeavyWord tokens)
    int32_t *heavy_row = nullptr;
    uint32_t *heavy_hist = nullptr;
    int n_heavy = 0;
    std::vector<pulda::HeavyChunk> heavy_chunks;     // host copy (chain 0)
    pulda::HeavyChunk *d_heavy_chunks = nullptr;
    pulda::PhiArgs *d_self = nullptr;         // this chain's PhiArgs on the device (for the heavy pass)
};


namespace pulda {
// Device memory through the caller's allocator (o.alloc / o.free) when set,
// else cudaMallocAsync / cudaFreeAsync on st (stream_ordered) or cudaMalloc /
// cudaFree.  A NULL or misaligned pointer from the caller's allocator is
// cudaErrorMemoryAllocation / cudaErrorMisalignedAddress (the latter given
// back first).
cudaError_t dev_alloc(const pulda_options &o, cudaStream_t st, size_t bytes, void **out, bool stream_ordered);
void dev_free(const pulda_options &o, cudaStream_t st, void *p, bool stream_ordered);
// A temporary device buffer of a call, given back (stream-ordered) when the
// call returns, on success or failure alike.
struct DevTemp {
    const pulda_options *o;
    cudaStream_t st;
    void *p = nullptr;
    DevTemp(const pulda_options &opt, cudaStream_t s) : o(&opt), st(s) {}
    DevTemp(const DevTemp &) = delete;
    DevTemp &operator=(const DevTemp &) = delete;
    ~DevTemp() { dev_free(*o, st, p, true); }
    template <typename T>
    cudaError_t get(T **out, size_t count) {
        cudaError_t e = dev_alloc(*o, st, sizeof(T) * (count > 0 ? count : 1), &p, true);
        *out = static_cast<T *>(p);
        return e;
    }
};
PhiArgs phi_args(pulda_handle *h);
ZArgs z_args(pulda_handle *h, const int64_t *doc_off, const int32_t *doc_order, int64_t D, const int32_t *w,
             int16_t *z, uint64_t seed, uint32_t sweep, int64_t index_base);
}  // namespace pulda
