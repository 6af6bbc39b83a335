// CUDA kernels of the Polya-urn partially collapsed LDA sampler, sm_103a.
//
// One sweep = Algorithm 2 (Section 3):
//   Phi-step  k_heavy_hist   words with more than 2^17 tokens histogrammed in
//                            chunks by many CTAs.
//             k_phi_counts   per word v: rebuild n_{.,v} from z (shared-memory
//                            histogram over the word's tokens), draw
//                            c_{k,v} ~ Pois(beta + n_{k,v}) for every k (Eq. 9,
//                            "Efficient sampling of Phi"), accumulate S_k.
//             k_phi_fixup    rows with S_k = 0 are redrawn until nonzero
//                            (Definition "Poisson Polya Urn").
//             k_scan_single  column offsets of the sparse Phi.
//             k_phi_tables   phi = c/S, fixed-point weights, sigma_a, the
//                            per-word alias table, bitmaps and dense q rows
//                            ("Efficient sampling of z").
//   z-step    k_z_step       one warp per document, tokens in order, the
//                            doubly sparse a/b draw (k_slice_counts first
//                            when long documents run in stale-count slices).
// The *_multi kernels do the same over many chains; k_serve_step folds in
// requests; the longest documents go to the cooperative z-step (one CTA per
// document, coop.cu); Algorithm 1's Dirichlet Phi-step is in dirichlet.cu.
// The arithmetic that decides any draw is integer or IEEE double with
// explicit rounding, so results are independent of launch shapes.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <type_traits>

#include "device_rng.cuh"
#include "pulda_internal.h"
#include "zstep.cuh"
#include "checks.cuh"

namespace pulda {
namespace {



// ------------------------------------------------------- Phi-step draws
// Alias-table draw from table t: slot floor(xs * n / 2^32), kept if xa < thr.
__device__ __forceinline__ uint32_t table_draw(const DevTables &T, int t, uint32_t xs, uint32_t xa) {
    const int off = T.off[t];
    const uint32_t s = __umulhi(xs, static_cast<uint32_t>(T.n[t]));
    const uint32_t j = xa < T.thr[off + s] ? s : static_cast<uint32_t>(T.alias[off + s]);
    return static_cast<uint32_t>(T.lo[t] + static_cast<int>(j));
}

// c ~ Pois(beta + l) for l >= 1: alias table for l <= L, rounded Gaussian
// mu + sqrt(mu) g, mu = beta + l, above.  g is interpolated linearly inside
// one of 2^16 equiprobable cells of the normal law.
__device__ uint32_t draw_entry(const DevTables &T, uint32_t l, uint32_t x0, uint32_t x1) {
    if (l <= static_cast<uint32_t>(kL)) return table_draw(T, static_cast<int>(l), x0, x1);
    const double g = gauss_draw(T, x0, x1);
    const double mu = __dadd_rn(T.beta, static_cast<double>(l));
    const double sd = __dsqrt_rn(mu);
    double r = floor(__dadd_rn(__dadd_rn(mu, __dmul_rn(sd, g)), 0.5));
    if (r < 0.0) r = 0.0;
    if (r > 4294967295.0) r = 4294967295.0;
    return static_cast<uint32_t>(r);
}

// Smallest g with x < geo[g]; -1 when the gap is at least kGeoLen.
__device__ __forceinline__ int geo_gap(const uint32_t *geo, uint32_t x) {
    if (x >= geo[kGeoLen - 1]) return -1;
    int lo = 0, hi = kGeoLen - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (x < geo[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// ------------------------------------------------------- block helpers
template <int BLOCK>
__device__ __forceinline__ int block_excl_scan(int v, int *tmp /* >= BLOCK/32 + 1 */, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < BLOCK / 32 ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < BLOCK / 32) tmp[lane] = t;
    }
    __syncthreads();
    total = tmp[BLOCK / 32 - 1];
    const int base = warp ? tmp[warp - 1] : 0;
    __syncthreads();
    return base + x - v;
}

// ================================================================= init
__global__ void k_init_z(int64_t N, int K, uint64_t seed, int64_t base, int16_t *z) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint64_t t = static_cast<uint64_t>(base + i);
        const U4 x = draw(seed, static_cast<uint32_t>(t), static_cast<uint32_t>(t >> 32), 0, TAG_INIT, 0);
        z[i] = static_cast<int16_t>(__umulhi(x.x, static_cast<uint32_t>(K)));
    }
}

// word-major permutation: counting sort of token ids by word id
__global__ void k_word_hist(int64_t N, const int32_t *w, int32_t *cnt) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&cnt[w[i]], 1);
}

// Exclusive scan of cnt[0..n) into out[0..n] (out[n] = total), one block.
template <typename TIn>
__global__ void k_scan_single(const TIn *cnt, int64_t n, int64_t *out, unsigned long long *total_slot) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t a = t * per, b = min(n, a + per);
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int i = 0; i < static_cast<int>(blockDim.x); ++i) { const int64_t v = part[i]; part[i] = run; run += v; }
        out[n] = run;
        if (total_slot) *total_slot = static_cast<unsigned long long>(run);
    }
    __syncthreads();
    int64_t run = part[t];
    for (int64_t i = a; i < b; ++i) { out[i] = run; run += cnt[i]; }
}

__global__ void k_word_scatter(int64_t N, const int32_t *w, const int64_t *word_off, int32_t *fill, int32_t *perm) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int v = w[i];
        const int pos = atomicAdd(&fill[v], 1);
        perm[word_off[v] + pos] = static_cast<int32_t>(i);
    }
}

// ======================================================== Phi-step: counts
constexpr int kPhiBlock = 256;
#ifndef PULDA_PHI_COUNT_BLOCK
#define PULDA_PHI_COUNT_BLOCK 128
#endif
constexpr int kPhiCountBlock = PULDA_PHI_COUNT_BLOCK;

// Sweep counter of a chain: from device memory when the launch is replayed
// from a CUDA graph (one graph serves every sweep), else the launch value.
__device__ __forceinline__ uint32_t sweep_of(const PhiArgs &a) { return a.sweep_ptr ? *a.sweep_ptr : a.sweep; }

// Adds the topics of the word-ordered tokens [b, e) into hist (shared
// memory), by a CTA of BLOCK threads.  The topics are gathered through perm
// from all over the corpus, so each thread issues kHistBatch of those loads
// before the first atomic: latency, not bandwidth, bounds a loop that waits
// on one at a time.
#ifndef PULDA_HIST_BATCH
#define PULDA_HIST_BATCH 8
#endif
constexpr int kHistBatch = PULDA_HIST_BATCH;
template <int BLOCK>
__device__ __forceinline__ void hist_tokens(const PhiArgs &a, int64_t b, int64_t e, uint32_t *hist) {
    const int K = a.K;
    int64_t t = b + threadIdx.x;
    for (; t + (kHistBatch - 1) * BLOCK < e; t += kHistBatch * BLOCK) {
        int32_t p[kHistBatch];
        int zz[kHistBatch];
#pragma unroll
        for (int u = 0; u < kHistBatch; ++u) p[u] = a.perm[t + u * BLOCK];
#pragma unroll
        for (int u = 0; u < kHistBatch; ++u) zz[u] = a.z[p[u]];
#pragma unroll
        for (int u = 0; u < kHistBatch; ++u) atomicAdd(&hist[guard_index(zz[u], K, a.stats)], 1u);
    }
    for (; t < e; t += BLOCK) atomicAdd(&hist[guard_index(a.z[a.perm[t]], K, a.stats)], 1u);
}

// One word v of one chain, by the whole CTA of BLOCK threads: histogram of
// the word's topics -> n_{.,v}; compacted n column; when `draw`, the Poisson
// draws c_{.,v}, the compacted c column, and S_k += c_{k,v}.  hist/cbin hold
// K entries each.  With `next` set, thread 0 takes the CTA's next work item
// from `work` once every thread is past reading the current one; the last
// barrier publishes it.
template <int BLOCK>
__device__ void phi_word(const PhiArgs &a, int v, bool do_draw, uint32_t *hist, uint32_t *cbin, int *scan_tmp,
                         const uint32_t *geo, int *next = nullptr, int *work = nullptr) {
    const int K = a.K;
    const uint32_t sweep = sweep_of(a);
    const int per = (K + BLOCK - 1) / BLOCK;     // bins owned by each thread, contiguous
    const int64_t wbeg = a.word_off[v], wend = a.word_off[v + 1];
    const int hrow = a.heavy_row ? a.heavy_row[v] : -1;
    if (a.counted) {
        // the n column was built by the sort path (countsort.cu)
        for (int k = threadIdx.x; k < K; k += BLOCK) { hist[k] = 0; cbin[k] = 0; }
        __syncthreads();
        const int nn = a.nnz_n[v];
        for (int j = threadIdx.x; j < nn; j += BLOCK)
            hist[guard_index(a.nst_k[wbeg + j], K, a.stats)] = a.nst_n[wbeg + j];
        __syncthreads();
    } else if (hrow >= 0) {
        const uint32_t *hh = a.heavy_hist + static_cast<int64_t>(hrow) * K;   // from L2: just summed by other CTAs
        for (int k = threadIdx.x; k < K; k += BLOCK) { hist[k] = __ldcg(&hh[k]); cbin[k] = 0; }
        __syncthreads();
    } else {
        for (int k = threadIdx.x; k < K; k += BLOCK) { hist[k] = 0; cbin[k] = 0; }
        __syncthreads();
        hist_tokens<BLOCK>(a, wbeg, wend, hist);
        __syncthreads();
    }
    if (next && threadIdx.x == 0) *next = atomicAdd(work, 1);
    if (do_draw) {
        // entries with n_{k,v} = l >= 1: c ~ Pois(beta + l)
        for (int k = threadIdx.x; k < K; k += BLOCK) {
            const uint32_t l = hist[k];
            if (l) {
                const U4 x = draw(a.seed, static_cast<uint32_t>(v), static_cast<uint32_t>(k), sweep, TAG_POIS, 0);
                cbin[k] = draw_entry(a.tab, l, x.x, x.y);
            }
        }
        // entries with n_{k,v} = 0: Pois(beta) by geometric skip-ahead.  The
        // walk's draws h = 0, 1, ... do not depend on where it stands, so
        // warp 0 draws 32 of them at once and a prefix sum of the gaps places
        // them -- the same hits, in the same order, as one thread walking.
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int pos = -1;
            for (uint32_t h0 = 0;; h0 += 32) {
                const U4 x = draw(a.seed, static_cast<uint32_t>(v), h0 + lane, sweep, TAG_BETA, 0);
                const int g = geo_gap(geo, x.x);
                const int step = g < 0 ? kGeoLen : g + 1;      // positions advanced by this draw
                int incl = step;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int p = pos + incl;                       // the hit's position (or where a skip ends)
                const bool stop = g < 0 ? p >= K - 1 : p >= K;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, stop);
                const int first_stop = bal ? __ffs(bal) - 1 : 32;
                if (lane < first_stop && g >= 0 && hist[p] == 0) cbin[p] = table_draw(a.tab, 0, x.y, x.z);
                if (bal) break;
                pos = __shfl_sync(0xFFFFFFFFu, p, 31);
            }
        }
        __syncthreads();
    }
    // compaction in ascending topic order
    const int k0 = threadIdx.x * per, k1 = min(K, k0 + per);
    int cn = 0, cc = 0;
    for (int k = k0; k < k1; ++k) { cn += hist[k] != 0; cc += cbin[k] != 0; }
    // one scan of both counts, n's in the low and c's in the high 16 bits
    // (each at most K <= 16384)
    int tboth;
    const int pboth = block_excl_scan<BLOCK>(cn | (cc << 16), scan_tmp, tboth);
    int pn = pboth & 0xFFFF, pc = pboth >> 16;
    const int tn = tboth & 0xFFFF, tc = tboth >> 16;
    for (int k = k0; k < k1; ++k) {
        const uint32_t l = hist[k];
        if (l) { a.nst_k[wbeg + pn] = static_cast<uint16_t>(k); a.nst_n[wbeg + pn] = l; ++pn; }
        if (do_draw) {
            const uint32_t c = cbin[k];
            if (c) {
                const int64_t o = static_cast<int64_t>(v) * K + pc;
                a.cst_k[o] = static_cast<uint16_t>(k);
                a.cst_c[o] = c;
                atomicAdd(&a.S[k], static_cast<u64>(c));
                ++pc;
            }
        }
    }
    if (threadIdx.x == 0) {
        a.nnz_n[v] = tn;
        if (do_draw) a.nnz_c[v] = tc;
    }
    __syncthreads();
}

// One chain's words, dynamically scheduled, most frequent first; CTAs of
// kPhiCountBlock threads (more words in flight per SM than 256-thread CTAs;
// a word's barriers then wait on fewer warps).
__global__ void __launch_bounds__(kPhiCountBlock) k_phi_counts(PhiArgs a, bool do_draw) {
    extern __shared__ uint32_t sm[];
    __shared__ int scan_tmp[kPhiCountBlock / 32 + 1];
    __shared__ int s_item;
    __shared__ uint32_t geo[kGeoLen];
    for (int i = threadIdx.x; i < kGeoLen; i += kPhiCountBlock) geo[i] = a.tab.geo[i];
    if (threadIdx.x == 0) s_item = atomicAdd(a.work, 1);
    __syncthreads();
    for (;;) {
        const int item = s_item;      // published by the barrier above, then by phi_word's last one
        if (item >= a.V) break;
        phi_word<kPhiCountBlock>(a, a.word_order[item], do_draw, sm, sm + a.K, scan_tmp, geo, &s_item, a.work);
    }
}

// Many chains: the work list holds (chain, word) pairs, most frequent first
// across all chains; shared memory is sized for the largest K.
__global__ void __launch_bounds__(kPhiBlock) k_phi_counts_multi(const PhiArgs *chains, const int2 *items,
                                                                 int n_items, int *work, int kmax, bool do_draw) {
    extern __shared__ uint32_t sm[];
    __shared__ int scan_tmp[kPhiBlock / 32 + 1];
    __shared__ int s_item;
    __shared__ uint32_t geo[kGeoLen];
    int geo_chain = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const int2 it = items[item];
        if (it.x != geo_chain) {          // the geometric table depends on the chain's beta
            for (int i = threadIdx.x; i < kGeoLen; i += kPhiBlock) geo[i] = chains[it.x].tab.geo[i];
            geo_chain = it.x;
            __syncthreads();
        }
        phi_word<kPhiBlock>(chains[it.x], it.y, do_draw, sm, sm + kmax, scan_tmp, geo);
    }
}

// Topic histograms of the most frequent words, one chunk of a word's tokens
// per CTA, added into the word's row of heavy_hist (zeroed before).
__device__ void heavy_chunk(const PhiArgs *chains, const HeavyChunk &c, uint32_t *hs) {
    const PhiArgs &a = chains[c.chain];
    const int K = a.K;
    for (int k = threadIdx.x; k < K; k += kPhiBlock) hs[k] = 0;
    __syncthreads();
    hist_tokens<kPhiBlock>(a, c.begin, c.end, hs);
    __syncthreads();
    uint32_t *row = a.heavy_hist + static_cast<int64_t>(c.row) * K;
    for (int k = threadIdx.x; k < K; k += kPhiBlock)
        if (hs[k]) atomicAdd(&row[k], hs[k]);
    __syncthreads();
}

__global__ void __launch_bounds__(kPhiBlock) k_heavy_hist(const PhiArgs *chains, const HeavyChunk *chunks, int kmax) {
    extern __shared__ uint32_t hs[];
    heavy_chunk(chains, chunks[blockIdx.x], hs);
    (void)kmax;
}

// n_{k,v} from the compacted n column of word v (binary search), 0 if absent.
__device__ uint32_t lookup_n(const PhiArgs &a, int v, int k) {
    const int64_t b = a.word_off[v];
    int lo = 0, hi = a.nnz_n[v];
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int km = a.nst_k[b + mid];
        if (km < k) lo = mid + 1; else hi = mid;
    }
    return (lo < a.nnz_n[v] && a.nst_k[b + lo] == k) ? a.nst_n[b + lo] : 0u;
}

constexpr int kFixBlock = 1024;

// Rows whose Poisson counts summed to zero are redrawn whole (attempt
// a = 1, 2, ...) until the sum is nonzero: the urn total is Pois+ (the
// hierarchical representation, Eq. 8).  Accepted rows are inserted into the
// word columns.  One block of BLOCK threads; almost always just checks S and
// exits.  S is read from L2 (other CTAs of the same launch may have just
// summed it).
template <int BLOCK>
__device__ void phi_fixup_chain(const PhiArgs &a, u64 *red, u64 *s_sum_p) {
    u64 &s_sum = *s_sum_p;
    const uint32_t sweep = sweep_of(a);
    // almost always no row is dead: one parallel look at S first
    int dead = 0;
    for (int k = threadIdx.x; k < a.K; k += BLOCK) dead |= __ldcg(&a.S[k]) == 0 ? 1 : 0;
    if (!__syncthreads_or(dead)) return;
    for (int k = 0; k < a.K; ++k) {
        if (__ldcg(&a.S[k]) != 0) continue;
        if (threadIdx.x == 0) atomicAdd(&a.stats[ST_DEADROWS], 1ull);
        uint32_t att = 1;
        for (; att <= kMaxRedraw; ++att) {
            u64 part = 0;
            for (int v = threadIdx.x; v < a.V; v += BLOCK) {
                const uint32_t l = lookup_n(a, v, k);
                uint32_t val = 0;
                if (l) {
                    const U4 x = draw(a.seed, static_cast<uint32_t>(v), static_cast<uint32_t>(k), sweep, TAG_REDRAW_POIS, att);
                    val = draw_entry(a.tab, l, x.x, x.y);
                }
                a.rowbuf[v] = val;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int64_t pos = -1;
                uint32_t h = 0;
                for (;;) {
                    const U4 x = draw(a.seed, static_cast<uint32_t>(k), h++, sweep, TAG_REDRAW_BETA, att);
                    const int g = geo_gap(a.tab.geo, x.x);
                    if (g < 0) {
                        pos += kGeoLen;
                        if (pos >= a.V - 1) break;
                        continue;
                    }
                    pos += g + 1;
                    if (pos >= a.V) break;
                    if (lookup_n(a, static_cast<int>(pos), k) == 0) a.rowbuf[pos] = table_draw(a.tab, 0, x.y, x.z);
                }
            }
            __syncthreads();
            for (int v = threadIdx.x; v < a.V; v += BLOCK) part += a.rowbuf[v];
            part = warp_sum64(part);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
            __syncthreads();
            if (threadIdx.x == 0) {
                u64 s = 0;
                for (int i = 0; i < BLOCK / 32; ++i) s += red[i];
                s_sum = s;
            }
            __syncthreads();
            const u64 sum = s_sum;
            if (sum > 0) {
                for (int v = threadIdx.x; v < a.V; v += BLOCK) {
                    const uint32_t val = a.rowbuf[v];
                    if (!val) continue;
                    const int64_t base = static_cast<int64_t>(v) * a.K;
                    int n = a.nnz_c[v];
                    int p = n;
                    while (p > 0 && a.cst_k[base + p - 1] > k) {
                        a.cst_k[base + p] = a.cst_k[base + p - 1];
                        a.cst_c[base + p] = a.cst_c[base + p - 1];
                        --p;
                    }
                    a.cst_k[base + p] = static_cast<uint16_t>(k);
                    a.cst_c[base + p] = val;
                    a.nnz_c[v] = n + 1;
                }
                if (threadIdx.x == 0) a.S[k] = sum;
                __syncthreads();
                break;
            }
            __syncthreads();
        }
        if (att > kMaxRedraw) {
            if (threadIdx.x == 0) atomicOr(&a.stats[ST_ERROR], ERR_DEGENERATE);
            return;
        }
    }
}

__global__ void __launch_bounds__(kFixBlock) k_phi_fixup(PhiArgs a) {
    __shared__ u64 red[kFixBlock / 32];
    __shared__ u64 s_sum;
    phi_fixup_chain<kFixBlock>(a, red, &s_sum);
}

// Many chains: one CTA per chain.
__global__ void __launch_bounds__(kFixBlock) k_phi_fixup_multi(const PhiArgs *chains) {
    __shared__ u64 red[kFixBlock / 32];
    __shared__ u64 s_sum;
    phi_fixup_chain<kFixBlock>(chains[blockIdx.x], red, &s_sum);
}

// Column offsets of one chain's Phi by one CTA (part: blockDim entries).
__device__ void colptr_chain(const PhiArgs &a, int64_t *part) {
    const int t = threadIdx.x;
    const int64_t n = a.V;
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = t * per, hi = min(n, lo + per);
    int64_t sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += a.nnz_c[i];
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int i = 0; i < static_cast<int>(blockDim.x); ++i) { const int64_t v = part[i]; part[i] = run; run += v; }
        a.col_ptr[n] = run;
        a.stats[ST_NNZPHI] = static_cast<unsigned long long>(run);
    }
    __syncthreads();
    int64_t run = part[t];
    for (int64_t i = lo; i < hi; ++i) { a.col_ptr[i] = run; run += a.nnz_c[i]; }
    __syncthreads();
}

// Column offsets of every chain's Phi: one CTA per chain.
__global__ void k_colptr_scan_multi(const PhiArgs *chains) {
    __shared__ int64_t part[1024];
    colptr_chain(chains[blockIdx.x], part);
}

// =================================================== Phi-step: tables
// Per word: phi = fp32(c/S) (Dirichlet mode: gamma (1/S), over the entries
// the selection kept); fixed-point weights q with
// 24 bits relative to the column maximum (q >= 1); alpha-part masses
// a = round(q alpha 2^16), A = sigma_a; Vose alias table over a; bitmap of
// the word's nonzero topics.
// The same per-word tables, one warp per word: the per-entry arithmetic in
// parallel, the Vose pairing (sequential by definition) in lane 0.
__device__ void phi_tables_word_warp(const PhiArgs &a, int v) {
    const int lane = threadIdx.x & 31;
    const int n = a.nnz_c[v];
    const int64_t src = static_cast<int64_t>(v) * a.K;
    const int64_t out = a.col_ptr[v];
    if (a.bits) {
        // a row of KWp words (KW rounded up; the words past KW stay zero)
        uint32_t *bm = a.bits + static_cast<int64_t>(v) * a.KWp;
        for (int wi = lane; wi < a.KWp; wi += 32) {
            int lo = 0, hi = n;                       // first entry with topic >= 32 wi
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (a.cst_k[src + mid] < 32 * wi) lo = mid + 1; else hi = mid; }
            uint32_t bits = 0;
            for (int j = lo; j < n && (a.cst_k[src + j] >> 5) == wi; ++j) bits |= 1u << (a.cst_k[src + j] & 31);
            bm[wi] = bits;
        }
    }
    // a word with a dense q row: zero it (the column's entries are written below)
    uint32_t *qrow = nullptr;
    if (a.dense_slot) {
        const int slot = a.dense_slot[v];
        if (slot >= 0) {
            qrow = a.qdense + static_cast<int64_t>(slot) * a.K;
            for (int k = lane; k < a.K; k += 32) qrow[k] = 0;
            __syncwarp();
        }
    }
    if (n == 0) {
        if (lane == 0) a.A[v] = 0;
        return;
    }
    double phimax = 0.0;
    for (int j = lane; j < n; j += 32) {
        const int k = a.cst_k[src + j];
        // Polya urn: c / S_k; Dirichlet: gamma (1 / S_k), gamma's float bits staged in cst_c
        const double p = a.gam ? __dmul_rn(static_cast<double>(__uint_as_float(a.cst_c[src + j])), a.invS[k])
                               : __ddiv_rn(static_cast<double>(a.cst_c[src + j]), static_cast<double>(__ldcg(&a.S[k])));
        a.vose_p[out + j] = static_cast<u64>(__double_as_longlong(p));    // phi, kept for the second pass
        phimax = p > phimax ? p : phimax;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double y = __shfl_xor_sync(0xFFFFFFFFu, phimax, o);
        phimax = y > phimax ? y : phimax;
    }
    // phimax = f 2^e with f in [1/2, 1); scale = 2^(24 - e) (exact)
    const long long bits = __double_as_longlong(phimax);
    const int e = static_cast<int>((bits >> 52) & 0x7FF) - 1022;
    const double scale = __longlong_as_double(static_cast<long long>(1023 + 24 - e) << 52);
    u64 asum = 0;
    for (int j = lane; j < n; j += 32) {
        const int k = a.cst_k[src + j];
        const uint32_t c = a.cst_c[src + j];
        const double p = __longlong_as_double(static_cast<long long>(a.vose_p[out + j]));
        const double qq = floor(__dadd_rn(__dmul_rn(p, scale), 0.5));
        const uint32_t qv = qq < 1.0 ? 1u : static_cast<uint32_t>(qq);
        const double at = __dmul_rn(__dmul_rn(static_cast<double>(qv), static_cast<double>(a.alpha[k])), 65536.0);
        const u64 am = static_cast<u64>(floor(__dadd_rn(at, 0.5)));
        a.topic[out + j] = static_cast<uint16_t>(k);
        a.c[out + j] = c;
        a.q[out + j] = qv;
        if (qrow) qrow[k] = qv;
        a.vose_p[out + j] = am * static_cast<u64>(n);   // scaled so each slot holds A units
        a.athr[out + j] = 0xFFFFFFFFu;
        a.atopic[out + j] = static_cast<uint16_t>(k);
        if (a.apack) a.apack[out + j] = make_uint2(0xFFFFFFFFu, static_cast<uint32_t>(k) * 0x10001u);
        asum += am;
    }
    asum = warp_sum64(asum);
    if (lane == 0) a.A[v] = asum;
    __syncwarp();
    if (asum == 0) return;
    // Vose: small stack grows up from 0, large stack down from n-1, each in
    // ascending slot order.  The warp builds the two stacks with a ballot per
    // 32 slots; lane 0 pairs (sequential by definition); then every lane
    // computes the thresholds of its paired slots.
    // Thresholds floor(P 2^32 / A) divide by the word's invariant A:
    // Moller and Granlund's 2/1 division with a reciprocal of the normalised
    // divisor, one 128-bit division per word instead of one per slot (exact).
    const int sh = __clzll(static_cast<long long>(asum));
    const u64 dn = asum << sh;
    const u64 vinv = static_cast<u64>((~static_cast<unsigned __int128>(0)) / dn);   // floor((2^128-1)/dn) - 2^64
    u64 *P = a.vose_p + out;
    uint16_t *stk = a.vose_stack + out;
    int ns = 0, nl = 0;
    for (int j0 = 0; j0 < n; j0 += 32) {
        const int j = j0 + lane;
        const bool in = j < n;
        const bool small = in && P[j] < asum;
        const uint32_t bs = __ballot_sync(0xFFFFFFFFu, small), bl = __ballot_sync(0xFFFFFFFFu, in && !small);
        const uint32_t below = (1u << lane) - 1u;
        if (small) stk[ns + __popc(bs & below)] = static_cast<uint16_t>(j);
        else if (in) stk[n - 1 - (nl + __popc(bl & below))] = static_cast<uint16_t>(j);
        ns += __popc(bs);
        nl += __popc(bl);
    }
    __syncwarp();
    if (lane == 0) {
        while (ns > 0 && nl > 0) {
            const int s = stk[--ns];
            --nl;
            const int l = stk[n - 1 - nl];
            const u64 ps = P[s];             // final: s is not pushed again
            a.atopic[out + s] = a.topic[out + l];
            const u64 pl = P[l] - (asum - ps);
            P[l] = pl;
            if (pl < asum) stk[ns++] = static_cast<uint16_t>(l);
            else { stk[n - 1 - nl] = static_cast<uint16_t>(l); ++nl; }
        }
    }
    __syncwarp();
    // a paired slot's alias is another topic of the column; the rest keep
    // their own topic and threshold 2^32 - 1
    for (int j = lane; j < n; j += 32) {
        if (a.atopic[out + j] == a.topic[out + j]) continue;
        const u64 ps = P[j];
        // (u1, u0) = ps 2^32 2^sh, u1 < dn since ps < asum
        const u64 hi = ps >> 32, lo = ps << 32;
        const u64 u1 = sh ? (hi << sh) | (lo >> (64 - sh)) : hi;
        const u64 u0 = lo << sh;
        u64 q0 = vinv * u1;
        u64 q1 = __umul64hi(vinv, u1);
        const u64 t = q0 + u0;
        q1 += u1 + (t < q0 ? 1ull : 0ull);
        q0 = t;
        q1 += 1;
        u64 r = u0 - q1 * dn;
        if (r > q0) { q1 -= 1; r += dn; }
        if (r >= dn) q1 += 1;
        a.athr[out + j] = static_cast<uint32_t>(q1);
        if (a.apack)
            a.apack[out + j] = make_uint2(static_cast<uint32_t>(q1),
                                          a.topic[out + j] | (static_cast<uint32_t>(a.atopic[out + j]) << 16));
    }
}

// One warp per word, most frequent first (their columns are the longest).
__global__ void k_phi_tables(PhiArgs a) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = wid; i < a.V; i += nwarps) phi_tables_word_warp(a, a.word_order[i]);
}

__global__ void k_phi_tables_multi(const PhiArgs *chains, const int2 *items, int n_items) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = wid; i < n_items; i += nwarps) {
        const int2 it = items[i];
        phi_tables_word_warp(chains[it.x], it.y);
    }
}

// ============================================================== z-step
// Entries of the document-side intersection each lane gathers with
// independent loads before consuming them.
#ifndef PULDA_ZGATHER
#define PULDA_ZGATHER 7
#endif
// 4-warp CTAs, 8 per SM: the kernel fits 64 registers without
// spilling and 32 warps share each SM (issue slots are what bound it; fewer
// warps leave them idle while each warp waits on its dependent chain).
#ifndef PULDA_ZMINBLOCKS
#define PULDA_ZMINBLOCKS 8
#endif
constexpr int kGather = PULDA_ZGATHER;
// the same for 16 and 8 topics per lane (fewer bits per lane)
#ifndef PULDA_ZGATHER16
#define PULDA_ZGATHER16 5
#endif
#ifndef PULDA_ZGATHER8
#define PULDA_ZGATHER8 4
#endif
constexpr int kGather16 = PULDA_ZGATHER16;
constexpr int kGather8 = PULDA_ZGATHER8;

// Index of topic k's count with TPL topics per lane: a gap word after each
// lane's TPL slots keeps the lanes' slots on distinct banks.
template <int TPL>
__device__ __forceinline__ int mit(int k) { return k + k / TPL; }

// A lane's bits of its TPL topics: 32 bits, or 64 for 64 topics per lane.
template <int TPL>
using lane_word_t = typename std::conditional<TPL == 64, uint64_t, uint32_t>::type;

// This lane's TPL bits of a bitmap row starting at word `row`.
template <int TPL>
__device__ __forceinline__ lane_word_t<TPL> lane_bits(const uint32_t *bits, int64_t row, int lane) {
    if constexpr (TPL == 64) {
        const uint32_t *p = bits + row + 2 * lane;
        return static_cast<uint64_t>(p[0]) | (static_cast<uint64_t>(p[1]) << 32);
    } else if constexpr (TPL == 32) {
        return bits[row + lane];
    } else {
        const uint32_t w = bits[row + (lane * TPL >> 5)];
        return (w >> ((lane * TPL) & 31)) & ((1u << (TPL & 31)) - 1u);
    }
}

// 1 << b in a lane word, 0 for b = -1.
template <int TPL>
__device__ __forceinline__ lane_word_t<TPL> lane_bit(int b) {
    if constexpr (TPL == 64) return bit_or_zero64(b);
    else return bit_or_zero(b);
}

// 1 << b in a lane word for b in [0, TPL).
template <int TPL>
__device__ __forceinline__ lane_word_t<TPL> lane_bit_at(int b) {
    return static_cast<lane_word_t<TPL>>(1) << b;
}

__device__ __forceinline__ int popc_word(uint32_t x) { return __popc(x); }
__device__ __forceinline__ int popc_word(uint64_t x) { return __popcll(x); }

// One warp per document (dynamically scheduled, longest first).  m_d lives
// in shared memory as a dense count array; for K <= 2048 each lane also holds
// the bits of m_d's nonzero topics among the TPL it owns (TPL = 64 above 1024
// topics, 32, or 16 / 8 for K <= 512 / 256, so that small K still spreads
// over the warp), and the document side reads q of topic TPL lane + b from
// the word's dense q row.  Tokens are visited in position order: remove token i (m^{-i}),
// compute sigma_b = sum_k q_{k,v} m_k over the smaller of {k : m_k > 0} and
// {k : phi_{k,v} > 0} (complexity theorem), draw r = floor(u (A + 2^16 B)),
// take the alias draw if r < A, else the first topic where the running sum
// of q m passes (r - A) / 2^16; add the token back.
//
// Latency matters as much as throughput: a document's tokens are strictly
// sequential, so the longest documents bound the kernel.  Everything that
// depends only on the token (its word, Philox words, alias outcome, the
// word's bitmap) is fetched ahead; the only loads on the critical path are
// the q values of the intersection, issued together.
// Resamples the tokens of one document, by one warp, in position order,
// pass after pass, until `budget` tokens are done or `max_pass_end` passes
// have been completed.  m (K entries of shared memory) is rebuilt from the
// current topics first: with positions < pos already resampled in this pass
// that is exactly m of the sequential sampler at `pos`.  Returns the run's
// final (sweep, pos) through r.
// With m0 set, m starts from those K counts (a slice of a longer document,
// from the document's counts at the start of the pass) instead of the run's
// own topics.
template <int TPL, typename CT>
__device__ void z_doc_warp_t(const ZArgs &a, uint32_t *m, DocRun &r, u64 *wcnt, const uint32_t *m0) {
    static_assert(TPL == 8 || TPL == 16 || TPL == 32 || TPL == 64, "8, 16, 32 or 64 topics per lane");
    using BT = lane_word_t<TPL>;
    static_assert(sizeof(CT) == 2 || sizeof(CT) == 4, "16- or 32-bit counts");
    constexpr int kLead = 4 / static_cast<int>(sizeof(CT));    // counts before mt[0]: the leading zero's word
    constexpr int G = TPL >= 32 ? kGather : TPL == 16 ? kGather16 : kGather8;
    const int lane = threadIdx.x & 31;
    const int K = a.K;
    const bool use_bm = a.bits != nullptr && a.path != 1;
    if (r.len == 0 || r.budget <= 0) return;
    // Lane l owns topics [TPL l, TPL l + TPL) (TPL = 64, 32, 16 or 8 by K, so
    // that small K spreads over more lanes).  Topic k's count is
    // mt[mit<TPL>(k)]: lane l's topics sit at mt[(TPL + 1) l + b], and the word
    // before each lane's slots is a zero (mt[-1] for lane 0 and for the lanes
    // without topics, the gap word after lane l - 1's slots otherwise), so an
    // empty gather slot (bit -1) reads a zero count.  Counts are CT (16-bit
    // when every document of the launch is shorter than 2^16 tokens).
    CT *mt = reinterpret_cast<CT *>(m) + kLead;
    const int nl = TPL == 32 ? a.KW : (K + TPL - 1) / TPL;      // lanes that own topics
    const bool own = lane < nl;
    const int mo = own ? (TPL + 1) * lane : 0;   // this lane's count slots (document side)
    const int qo = own ? TPL * lane : 0;         // and its segment of a dense q row
    if (m0) {
        for (int k = lane; k < K; k += 32) mt[mit<TPL>(k)] = m0[k];
    } else {
        for (int k = lane; k < K; k += 32) mt[mit<TPL>(k)] = 0;
        __syncwarp();
        for (int i = lane; i < r.len; i += 32) {
            const int k = guard_index(r.z[i], K, a.stats);
            if (sizeof(CT) == 4) {
                atomicAdd(reinterpret_cast<uint32_t *>(&mt[mit<TPL>(k)]), 1u);
            } else {        // the 32-bit word holding the count: no carry, counts stay below 2^16
                const int h = mit<TPL>(k) + kLead;
                atomicAdd(m + (h >> 1), 1u << ((h & 1) * 16));
            }
        }
    }
    if (lane == 0) mt[-1] = 0;
    if (lane + 1 < nl) mt[(TPL + 1) * lane + TPL] = 0;
    __syncwarp();
    BT mbits = 0;
    int kd = 0;
    if (use_bm && TPL == 32) {
        for (int g = 0; g < a.KW; ++g) {
            const int k = g * 32 + lane;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, k < K && mt[mit<TPL>(k)] > 0);
            if (lane == g) mbits = bal;
            kd += __popc(bal);
        }
    } else if (use_bm) {
        if (own) {
            for (int b = 0; b < TPL; ++b) {
                const int k = TPL * lane + b;
                if (k < K && mt[mit<TPL>(k)] > 0) mbits |= lane_bit_at<TPL>(b);
            }
        }
        kd = static_cast<int>(__reduce_add_sync(0xFFFFFFFFu, static_cast<uint32_t>(popc_word(mbits))));
    } else {
        int cnt = 0;
        for (int k = lane; k < K; k += 32) cnt += mt[mit<TPL>(k)] > 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        kd = cnt;
    }
    // The run's state lives in the warp's shared memory while its tokens are
    // drawn (it is read and advanced once per 32-token block), which keeps it
    // out of the registers of the token loop.
    DocRun &rs = *z_warp_run(wcnt);
    if (lane == 0) rs = r;
    __syncwarp();
    const uint32_t sweep_end = rs.sweep + static_cast<uint32_t>(rs.max_pass_end);
    bool first = true;
    while (rs.budget > 0 && rs.sweep != sweep_end) {
        if (rs.deadline != ~0ull && !first) {
            uint64_t now = 0;
            if (lane == 0) now = global_ns();
            if (__shfl_sync(0xFFFFFFFFu, now, 0) >= rs.deadline) break;
        }
        first = false;
        const int i0 = rs.pos;
        const int64_t left = static_cast<int64_t>(rs.len - i0);
        const int cnt = static_cast<int>(min(static_cast<int64_t>(32), min(left, rs.budget)));
        const int i = i0 + lane;
        const bool valid = lane < cnt;
        int znew = 0;
        // Everything that depends only on the token is fetched for 32 tokens at
        // once, one per lane, and staged in shared memory:
        //   rec[2t]   = {column start (low 32), column start >> 32 | alias outcome << 16, sigma_a (lo, hi)}
        //   rec[2t+1] = {Philox x0, x1, word, K_v | old topic << 16}
        // (column starts are below 2^48, K_v <= 16384, topics < 16384).
        uint4 *rec = reinterpret_cast<uint4 *>(m + z_count_words<CT>(K));
        uint32_t *drow_of = reinterpret_cast<uint32_t *>(rec + 64);   // q row offset of the token's word, or ~0
        if (valid) znew = stage_token(a, rs, i, rec + 2 * lane, drow_of + lane);
        __syncwarp();
        // the word's bitmap row (TPL topics per lane)
        const uint32_t *bits = a.bits;
        BT bm_next = 0u;
        if (use_bm && own) bm_next = lane_bits<TPL>(bits, static_cast<int64_t>(rec[1].z) * a.KWp, lane);
        // this block's counters, in 32 bits (at most 32 tokens of K <= 16384),
        // added to the warp's 64-bit counters once per block
        // (c_min: sum of min(K_d, K_v), the same in every lane; c_cnt: tokens
        // with K_d < K_v in bits 0-5, alias draws in 6-11, zero-mass tokens in
        // 12-17 -- each at most 32 -- and this lane's share of |J| (at most
        // 32 x 32) from bit 18)
        uint32_t c_min = 0, c_cnt = 0;
        for (int tt = 0; tt < cnt; ++tt) {
            const uint4 t0 = rec[2 * tt], t1 = rec[2 * tt + 1];
            const int kold = static_cast<int>(t1.w >> 16);
            const int64_t col = static_cast<int64_t>((static_cast<u64>(t0.y & 0xFFFFu) << 32) | t0.x);
            const int n_w = static_cast<int>(t1.w & 0xFFFFu);
            const u64 At = (static_cast<u64>(t0.w) << 32) | t0.z;
            const u64 U = (static_cast<u64>(t1.x) << 32) | t1.y;
            const int ka = static_cast<int>(t0.y >> 16);
            const BT bm = bm_next;
            if (use_bm && tt + 1 < cnt && own)   // the next token's bitmap word, fetched while this one is drawn
                bm_next = lane_bits<TPL>(bits, static_cast<int64_t>(rec[2 * tt + 3].z) * a.KWp, lane);
            // remove token i: m^{-i}
            if (use_bm) {
                // the lane owning topic kold updates its count and bitmap word
                // (lanes read only their own counts on the document side)
                const bool me = lane == kold / TPL;
                const uint32_t old = me ? mt[mit<TPL>(kold)] : 0u;
                if (me) mt[mit<TPL>(kold)] = old - 1;
                const bool died = me && old == 1;
                if (died) mbits &= ~lane_bit_at<TPL>(kold % TPL);
                kd -= __any_sync(0xFFFFFFFFu, died) ? 1 : 0;
            } else {
                const uint32_t old = mt[mit<TPL>(kold)];
                __syncwarp();
                if (lane == 0) mt[mit<TPL>(kold)] = old - 1;
                if (old == 1) --kd;
                __syncwarp();
            }
            c_min += static_cast<uint32_t>(kd < n_w ? kd : n_w);
            c_cnt += kd < n_w ? 1u : 0u;
            // |J| from the bitmaps on either side (the column side's topics with
            // m > 0 are the same set); without bitmaps the column loop counts it
            if (use_bm) c_cnt += static_cast<uint32_t>(popc_word(bm & mbits)) << 18;
            // The document side needs the word's dense q row (q of topic TPL lane + b
            // at qd[b]); a word without one is iterated on the column side.
            const uint32_t drow = drow_of[tt];
            const bool docside = use_bm && drow != 0xFFFFFFFFu && (a.path == 2 || kd * kDocRatio < n_w * 16);
            const uint32_t *qcol = a.q + col;
            const uint32_t *qd = a.qdense + drow + qo;
            const CT *ml = mt + mo;
            // per-lane partial sums of q m, in ascending topic order across lanes
            u64 acc = 0;
            uint32_t qv[G];
            int bp[G];
            BT rest = 0;               // docside: bits below the first G
            int seg = 0, seg0 = 0;     // column side: this lane's contiguous segment
            if (docside) {
                // The lane's bits from the highest down; a slot past the last
                // bit gets b = -1 and q = 0 (no load), and its count read hits
                // the zero before the lane's slots.
                BT rem = bm & mbits;
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const int b = msb_or_neg1(rem);
                    rem ^= lane_bit<TPL>(b);
                    bp[t] = b;
                    qv[t] = b >= 0 ? qd[b] : 0u;
                }
#pragma unroll
                for (int t = 0; t < G; ++t) acc += static_cast<u64>(qv[t]) * ml[bp[t]];
                rest = rem;
                for (BT bb = rest; bb;) {
                    const int b = msb_or_neg1(bb);
                    bb ^= lane_bit<TPL>(b);
                    acc += static_cast<u64>(qd[b]) * ml[b];
                }
            } else {
                __syncwarp();   // the column side reads every lane's counts
                seg = (n_w + 31) >> 5;
                seg0 = seg * lane;
                const int seg1 = min(seg0 + seg, n_w);
                unsigned nj = 0;
#pragma unroll 4
                for (int j = seg0; j < seg1; ++j) {
                    const uint32_t mk = mt[mit<TPL>(guard_index(a.topic[col + j], K, a.stats))];
                    acc += static_cast<u64>(qcol[j]) * mk;
                    if (!use_bm) nj += mk != 0u;
                }
                if (!use_bm) c_cnt += nj << 18;
            }
            const u64 incl = warp_incl_scan64(acc);
            const u64 B = __shfl_sync(0xFFFFFFFFu, incl, 31);
            const u64 T = At + (B << kFracBits);
            int knew = kold;
            if (T == 0) {
                c_cnt += 1u << 12;
            } else {
                const u64 rr = __umul64hi(U, T);
                if (rr < At) {
                    knew = ka;
                    c_cnt += 1u << 6;
                } else {
                    const u64 rb = (rr - At) >> kFracBits;
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, rb < incl);
                    int found = -1;
                    if (bal) {
                        const int L = __ffs(bal) - 1;
                        int f = -1;
                        if (lane == L) {
                            if (docside) {
                                // walk down from the lane's inclusive sum: the
                                // topic whose term takes it to rb or below (an
                                // empty slot adds nothing, so the walk stops at
                                // one of the lane's bits)
                                u64 run = incl;
#pragma unroll
                                for (int t = 0; t < G; ++t) {
                                    run -= static_cast<u64>(qv[t]) * ml[bp[t]];
                                    if (rb >= run) { f = TPL * lane + bp[t]; break; }
                                }
                                for (BT bb = rest; f < 0 && bb;) {
                                    const int b = msb_or_neg1(bb);
                                    bb ^= lane_bit<TPL>(b);
                                    run -= static_cast<u64>(qd[b]) * ml[b];
                                    if (rb >= run) f = TPL * lane + b;
                                }
                            } else {
                                u64 run = incl - acc;
                                const int seg1 = min(seg0 + seg, n_w);
                                for (int j = seg0; j < seg1; ++j) {
                                    const int k = guard_index(a.topic[col + j], K, a.stats);
                                    run += static_cast<u64>(qcol[j]) * mt[mit<TPL>(k)];
                                    if (rb < run) { f = k; break; }
                                }
                            }
                        }
                        found = __shfl_sync(0xFFFFFFFFu, f, L);
                    }
                    if (found < 0) {
                        if (lane == 0) atomicOr(&a.stats[ST_ERROR], ERR_INTERNAL);
                    } else {
                        knew = found;
                    }
                }
            }
            // add token i back with its new topic
            knew = guard_index(knew, K, a.stats);
            if (use_bm) {
                const bool me = lane == knew / TPL;
                const uint32_t old2 = me ? mt[mit<TPL>(knew)] : 0u;
                if (me) mt[mit<TPL>(knew)] = old2 + 1;
                const bool born = me && old2 == 0;
                if (born) mbits |= lane_bit_at<TPL>(knew % TPL);
                kd += __any_sync(0xFFFFFFFFu, born) ? 1 : 0;
            } else {
                const uint32_t old2 = mt[mit<TPL>(knew)];
                __syncwarp();
                if (lane == 0) mt[mit<TPL>(knew)] = old2 + 1;
                if (old2 == 0) ++kd;
                __syncwarp();
            }
            if (lane == tt) znew = knew;
        }
        if (valid) rs.z[i] = static_cast<int16_t>(znew);
        {   // the block's counts into the warp's 64-bit counters, lane j its counter j
            const uint32_t jsum = __reduce_add_sync(0xFFFFFFFFu, c_cnt >> 18);
            const uint32_t v = lane == 0 ? static_cast<uint32_t>(cnt)
                             : lane == 1 ? (c_cnt >> 6) & 63u
                             : lane == 2 ? c_min
                             : lane == 3 ? (c_cnt >> 12) & 63u
                             : lane == 4 ? jsum : c_cnt & 63u;
            if (lane < 6) wcnt[lane] += v;
        }
        __syncwarp();
        if (lane == 0) {
            rs.budget -= cnt;
            rs.pos += cnt;
            if (rs.pos == rs.len) { rs.pos = 0; rs.sweep += 1; }
        }
        __syncwarp();
    }
    r = rs;
    __syncwarp();
}

// One chain, one document per warp (dynamically scheduled, longest first),
// one pass.
// TPL topics per lane (z_lane_topics(K)) and CT counts, one instantiation
// per kernel.
template <int TPL, typename CT>
__global__ void __launch_bounds__(32 * kZWarps, PULDA_ZMINBLOCKS) k_z_step(ZArgs a) {
    extern __shared__ uint32_t zsm[];
    const int lane = threadIdx.x & 31;
    uint32_t *m = zsm + static_cast<size_t>(threadIdx.x >> 5) * z_warp_words_t<CT>(a.K);
    u64 *wcnt = z_warp_counters_t<CT>(m, a.K);
    zero_warp_counters(wcnt);
    const uint32_t sweep = sweep_of(a);
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.work, 1);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item >= a.n_slices + a.D) break;
        int64_t s;
        int len;
        const uint32_t *m0 = nullptr;
        if (item < a.n_slices) {
            // a slice of a long document: {document, its row in m0, first token, tokens}
            const int4 sl = a.slices[item];
            s = a.doc_off[sl.x] + sl.z;
            len = sl.w;
            m0 = a.m0 + static_cast<int64_t>(sl.y) * a.K;
        } else {
            const int d = a.doc_order[item - a.n_slices];
            s = a.doc_off[d];
            len = static_cast<int>(a.doc_off[d + 1] - s);
        }
        DocRun r{a.w + s, a.z + s, len, a.seed, a.index_base + s, sweep, 0, len, 1};
        z_doc_warp_t<TPL, CT>(a, m, r, wcnt, m0);
    }
    flush_warp_counters(a.stats, wcnt);
}

// m0[j * K + k] = the topic-k count of document sliced_docs[j] (one warp per
// document): the pass-start counts its slices start from.
__global__ void k_slice_counts(const int64_t *doc_off, const int32_t *sliced_docs, int n, const int16_t *z, int K,
                               uint32_t *m0) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += nwarps) {
        uint32_t *row = m0 + static_cast<int64_t>(j) * K;
        for (int k = lane; k < K; k += 32) row[k] = 0;
        __syncwarp();
        const int d = sliced_docs[j];
        for (int64_t i = doc_off[d] + lane; i < doc_off[d + 1]; i += 32) atomicAdd(&row[z[i]], 1u);
        __syncwarp();
    }
}

// Many chains: the work list holds (chain, document) pairs, longest first
// across all chains; shared memory per warp is sized for the largest K.
// TPL = z_lane_topics(kmax): every chain of the batch that carries bitmaps has
// K <= kmax <= 32 TPL (the others iterate their columns);
// CT 16-bit when every document of every chain is shorter than 2^16 tokens.
template <int TPL, typename CT>
__global__ void __launch_bounds__(32 * kMultiWarps, PULDA_MULTI_MINB) k_z_step_multi(const ZArgs *chains, const int2 *items,
                                                                        int n_items, int *work, int kmax) {
    extern __shared__ uint32_t zsm[];
    const int lane = threadIdx.x & 31;
    uint32_t *m = zsm + static_cast<size_t>(threadIdx.x >> 5) * z_warp_words_t<CT>(kmax);
    u64 *wcnt = z_warp_counters_t<CT>(m, kmax);     // beyond every chain's m and token records
    zero_warp_counters(wcnt);
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(work, 1);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item >= n_items) break;
        const int2 it = items[item];
        const ZArgs &a = chains[it.x];
        const int64_t s = a.doc_off[it.y];
        DocRun r{a.w + s, a.z + s, static_cast<int>(a.doc_off[it.y + 1] - s), a.seed, a.index_base + s, sweep_of(a),
                 0, a.doc_off[it.y + 1] - s, 1};
        z_doc_warp_t<TPL, CT>(a, m, r, wcnt, nullptr);
        flush_warp_counters(a.stats, wcnt);
    }
}

// ============================================================ batches
// Start of a sweep of many chains (one CTA): advance the shared sweep counter
// and clear every chain's row sums, per-sweep counters and the work queues.
__device__ void batch_begin_sweep(const PhiArgs *chains, int n_chains, uint32_t *sweep, int *work) {
    if (threadIdx.x == 0) *sweep += 1u;
    if (threadIdx.x < 4) work[threadIdx.x] = 0;
    for (int c = 0; c < n_chains; ++c) {
        const PhiArgs &a = chains[c];
        for (int k = threadIdx.x; k < a.K; k += blockDim.x) a.S[k] = 0;
        for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x) a.stats[i] = 0;
        if (a.heavy_hist)
            for (int64_t i = threadIdx.x; i < static_cast<int64_t>(a.n_heavy) * a.K; i += blockDim.x) a.heavy_hist[i] = 0;
    }
}

__global__ void k_batch_begin_sweep(const PhiArgs *chains, int n_chains, uint32_t *sweep, int *work) {
    batch_begin_sweep(chains, n_chains, sweep, work);
}

// ============================================================ serving
// One step of the fold-in server: each active slot (a request's document,
// resampled with Phi fixed) advances by up to `slice` tokens, continuing
// across passes, one warp per slot.  A slot whose pass counter is 0 first
// gets its uniform initial topics (counter 0, as pulda_infer).  The slot's
// (pass, position) is written back for the host's completion check.
// Its slot bookkeeping needs a few more registers than k_z_step: 7 CTAs per
// SM keep it free of spills.
// With window_ns > 0 a slot also stops at the first 32-token block boundary
// window_ns after its warp took it up, having done at least one block (a slot
// taken up in a later wave of a crowded launch gets the same time as the first).
template <int TPL, typename CT>
__global__ void __launch_bounds__(32 * kZWarps, 7) k_serve_step(ZArgs a, ServeSlot *slots, const int32_t *active,
                                                                     int n_active, const int32_t *arena_w,
                                                                     int16_t *arena_z, int64_t slice, int *work,
                                                                     uint64_t window_ns) {
    extern __shared__ uint32_t zsm[];
    const int lane = threadIdx.x & 31;
    uint32_t *m = zsm + static_cast<size_t>(threadIdx.x >> 5) * z_warp_words_t<CT>(a.K);
    u64 *wcnt = z_warp_counters_t<CT>(m, a.K);
    zero_warp_counters(wcnt);
    for (;;) {
        int item = 0;
        uint64_t t0 = 0;
        if (lane == 0) {
            item = atomicAdd(work, 1);
            if (window_ns) t0 = global_ns();
        }
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item >= n_active) break;
        const uint64_t deadline = window_ns ? __shfl_sync(0xFFFFFFFFu, t0, 0) + window_ns : ~0ull;
        const int idx = active[item];
        const ServeSlot sl = slots[idx];
        int16_t *z = arena_z + sl.off;
        uint32_t sweep = sl.sweep;
        int pos = sl.pos;
        if (sweep == 0) {
            for (int i = lane; i < sl.len; i += 32) {
                const U4 x = draw(sl.seed, static_cast<uint32_t>(i), 0u, 0u, TAG_INIT, 0);
                z[i] = static_cast<int16_t>(__umulhi(x.x, static_cast<uint32_t>(a.K)));
            }
            __syncwarp();
            sweep = 1;
            pos = 0;
        }
        DocRun r{arena_w + sl.off, z, sl.len, sl.seed, 0, sweep, pos, slice,
                 static_cast<int>(sl.sweep_end - sweep), deadline};
        z_doc_warp_t<TPL, CT>(a, m, r, wcnt, nullptr);
        if (lane == 0) {
            slots[idx].sweep = r.sweep;
            slots[idx].pos = r.pos;
        }
    }
    flush_warp_counters(a.stats, wcnt);
}

// ============================================================== exports
// m_{d,k}, dense row-major [D, K]: one warp per document.
__global__ void k_doc_topic(const int64_t *doc_off, int64_t D, const int16_t *z, int K, int32_t *m_dk) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t d = gw; d < D; d += nw) {
        int32_t *row = m_dk + d * K;
        for (int64_t i = doc_off[d] + lane; i < doc_off[d + 1]; i += 32) atomicAdd(&row[z[i]], 1);
    }
}

// n_{k,v}, dense row-major [K, V], from the compacted n columns.
__global__ void k_n_dense(PhiArgs a, int32_t *n_kv) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < a.V; v += gridDim.x * blockDim.x) {
        const int64_t b = a.word_off[v];
        for (int j = 0; j < a.nnz_n[v]; ++j) n_kv[static_cast<int64_t>(a.nst_k[b + j]) * a.V + v] = static_cast<int32_t>(a.nst_n[b + j]);
    }
}

// phi_{k,v} = fp32(c_{k,v} / S_k) for every stored entry (Dirichlet mode:
// fp32(gamma_{k,v} (1 / S_k))).
__global__ void k_phi_values(PhiArgs a, float *phi) {
    const int64_t nnz = a.col_ptr[a.V];
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        phi[e] = a.gam ? static_cast<float>(__dmul_rn(static_cast<double>(__uint_as_float(a.c[e])), a.invS[a.topic[e]]))
                       : static_cast<float>(__ddiv_rn(static_cast<double>(a.c[e]), static_cast<double>(a.S[a.topic[e]])));
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

// ============================================================ launchers
void launch_init_z(int64_t N, int K, uint64_t seed, int64_t index_base, int16_t *z, cudaStream_t st) {
    if (N <= 0) return;
    const int grid = static_cast<int>(std::min<int64_t>((N + 255) / 256, 8LL * sm_count() * 8));
    k_init_z<<<grid, 256, 0, st>>>(N, K, seed, index_base, z);
}

void launch_word_perm(int64_t N, int V, const int32_t *w, int64_t *word_off, int32_t *fill, int32_t *perm,
                      cudaStream_t st) {
    cudaMemsetAsync(fill, 0, sizeof(int32_t) * V, st);
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 8LL * sm_count() * 8)));
    if (N > 0) k_word_hist<<<grid, 256, 0, st>>>(N, w, fill);
    k_scan_single<int32_t><<<1, 1024, 0, st>>>(fill, V, word_off, nullptr);
    cudaMemsetAsync(fill, 0, sizeof(int32_t) * V, st);
    if (N > 0) k_word_scatter<<<grid, 256, 0, st>>>(N, w, word_off, fill, perm);
}

size_t phi_counts_smem(int K) { return sizeof(uint32_t) * 2 * static_cast<size_t>(K); }

// The dynamic shared-memory opt-in is a per-kernel attribute shared by every
// handle in the process, so it is set once to the device maximum.
int smem_optin() {
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (v <= 0) v = 48 * 1024;
    }
    return v;
}

int phi_counts_blocks_per_sm(int K) {
    const size_t smem = phi_counts_smem(K);
    allow_dynamic_smem(k_phi_counts);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_phi_counts, kPhiCountBlock, smem);
    return b > 0 ? b : 1;
}

void launch_phi_counts(const PhiArgs &a, bool draw, int grid, cudaStream_t st) {
    const size_t smem = phi_counts_smem(a.K);
    k_phi_counts<<<grid, kPhiCountBlock, smem, st>>>(a, draw);
}

void launch_phi_fixup(const PhiArgs &a, cudaStream_t st) { k_phi_fixup<<<1, kFixBlock, 0, st>>>(a); }

void launch_colptr_scan(const PhiArgs &a, cudaStream_t st) {
    k_scan_single<int32_t><<<1, 1024, 0, st>>>(a.nnz_c, a.V, a.col_ptr, &a.stats[ST_NNZPHI]);
}

void launch_phi_tables(const PhiArgs &a, cudaStream_t st) {
    const int grid = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(a.V) * 32 + 255) / 256, 16LL * sm_count()));
    k_phi_tables<<<std::max(grid, 1), 256, 0, st>>>(a);
}

void launch_phi_tables_multi(const PhiArgs *chains, const int2 *items, int n_items, cudaStream_t st) {
    const int grid = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(n_items) * 32 + 255) / 256, 16LL * sm_count()));
    k_phi_tables_multi<<<std::max(grid, 1), 256, 0, st>>>(chains, items, n_items);
}

void launch_heavy_hist(const PhiArgs *chains, const HeavyChunk *chunks, int n_chunks, int kmax, cudaStream_t st) {
    if (n_chunks <= 0) return;
    static bool opted_in = false;
    if (!opted_in) { allow_dynamic_smem(k_heavy_hist); opted_in = true; }
    k_heavy_hist<<<n_chunks, kPhiBlock, sizeof(uint32_t) * static_cast<size_t>(kmax), st>>>(chains, chunks, kmax);
}

size_t z_step_smem(int K, int warps_per_block, bool narrow) {
    return sizeof(uint32_t) * static_cast<size_t>(z_warp_words_n(K, narrow)) * warps_per_block;
}

using ZStepKernel = void (*)(ZArgs);
static ZStepKernel z_step_kernel(int K, bool narrow) {
    switch (z_lane_topics(K)) {
        case 8: return narrow ? k_z_step<8, uint16_t> : k_z_step<8, uint32_t>;
        case 16: return narrow ? k_z_step<16, uint16_t> : k_z_step<16, uint32_t>;
        case 32: return narrow ? k_z_step<32, uint16_t> : k_z_step<32, uint32_t>;
        default: return narrow ? k_z_step<64, uint16_t> : k_z_step<64, uint32_t>;
    }
}

int z_step_blocks_per_sm(int K, int warps_per_block, bool narrow) {
    const size_t smem = z_step_smem(K, warps_per_block, narrow);
    ZStepKernel kern = z_step_kernel(K, narrow);
    allow_dynamic_smem(kern);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * warps_per_block, smem);
    return b > 0 ? b : 1;
}

void launch_slice_counts(const int64_t *doc_off, const int32_t *sliced_docs, int n, const int16_t *z, int K,
                         uint32_t *m0, cudaStream_t st) {
    if (n <= 0) return;
    const int grid = std::max(1, std::min((n + 7) / 8, 4 * sm_count()));
    k_slice_counts<<<grid, 256, 0, st>>>(doc_off, sliced_docs, n, z, K, m0);
}

void launch_z_step(const ZArgs &a, int warps_per_block, int grid, cudaStream_t st) {
    ZStepKernel kern = z_step_kernel(a.K, a.narrow != 0);
    // each instantiation opts in to large dynamic shared memory once
    static std::atomic<bool> opted[4][2];
    const int tpl = z_lane_topics(a.K);
    std::atomic<bool> &o = opted[tpl == 8 ? 0 : tpl == 16 ? 1 : tpl == 32 ? 2 : 3][a.narrow != 0];
    if (!o.load(std::memory_order_acquire)) {
        allow_dynamic_smem(kern);
        o.store(true, std::memory_order_release);
    }
    kern<<<grid, 32 * warps_per_block, z_step_smem(a.K, warps_per_block, a.narrow != 0), st>>>(a);
}

using ZMultiKernel = void (*)(const ZArgs *, const int2 *, int, int *, int);
static ZMultiKernel z_multi_kernel(int kmax, bool narrow) {
    switch (z_lane_topics(kmax)) {
        case 8: return narrow ? k_z_step_multi<8, uint16_t> : k_z_step_multi<8, uint32_t>;
        case 16: return narrow ? k_z_step_multi<16, uint16_t> : k_z_step_multi<16, uint32_t>;
        case 32: return narrow ? k_z_step_multi<32, uint16_t> : k_z_step_multi<32, uint32_t>;
        default: return narrow ? k_z_step_multi<64, uint16_t> : k_z_step_multi<64, uint32_t>;
    }
}

static void launch_z_step_multi(const BatchLaunch &b, const int2 *items, int n, cudaStream_t st) {
    ZMultiKernel kern = z_multi_kernel(b.kmax, b.narrow != 0);
    kern<<<b.z_grid, 32 * b.z_warps, z_step_smem(b.kmax, b.z_warps, b.narrow != 0), st>>>(b.z, items, n, b.work + 1,
                                                                                       b.kmax);
}

void launch_batch_sweep(const BatchLaunch &b, cudaStream_t st) {
    k_batch_begin_sweep<<<1, 256, 0, st>>>(b.phi, b.n_chains, b.sweep, b.work);
    launch_heavy_hist(b.phi, b.heavy, b.n_heavy, b.kmax, st);
    k_phi_counts_multi<<<b.phi_grid, kPhiBlock, phi_counts_smem(b.kmax), st>>>(b.phi, b.phi_items, b.n_phi_items,
                                                                                b.work, b.kmax, true);
    k_phi_fixup_multi<<<b.n_chains, kFixBlock, 0, st>>>(b.phi);
    k_colptr_scan_multi<<<b.n_chains, 1024, 0, st>>>(b.phi);
    launch_phi_tables_multi(b.phi, b.phi_items, b.n_phi_items, st);
    if (b.n_coop > 0) {
        // the longest documents on CTAs, the rest one per warp beside them
        cudaEventRecord(b.ev_fork, st);
        launch_z_step_coop_multi(b.z, b.z_items, b.n_coop, b.work + 2, b.kmax, b.coop_grid, st);
        cudaStreamWaitEvent(b.stream2, b.ev_fork, 0);
        if (b.n_z_items > b.n_coop)
            launch_z_step_multi(b, b.z_items + b.n_coop, b.n_z_items - b.n_coop, b.stream2);
        cudaEventRecord(b.ev_join, b.stream2);
        cudaStreamWaitEvent(st, b.ev_join, 0);
    } else {
        launch_z_step_multi(b, b.z_items, b.n_z_items, st);
    }
}

// ---------------------------------------------------------- one persistent launch per sweep
// The same sweep of many chains as launch_batch_sweep, in one cooperative
// launch whose CTAs are all resident: the phases (counter reset, heavy-word
// histograms, counts and draws, dead-row redraws, column offsets, per-word
// tables, z-step) run one after another, each over the whole grid, separated
// by a grid barrier.  Nothing a phase reads was read earlier in the launch by
// another SM before its writers finished (so no stale L1 line is read), except
// the row sums and heavy-word histograms, which are read from L2.
constexpr int kPersistThreads = 256;
constexpr int kPersistWarps = kPersistThreads / 32;
#ifndef PULDA_PERSIST_MINB
#define PULDA_PERSIST_MINB 4
#endif

// A grid barrier with a bounded wait: thread 0 of each CTA arrives; the last
// to arrive opens the next generation.  A CTA that has waited 2 s sets
// ERR_BARRIER in err and returns false (the launch then ends with an error
// instead of waiting forever).
__device__ bool grid_barrier(GridBarrier *bar, unsigned nblocks, unsigned long long *err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        volatile unsigned *gen = &bar->gen;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*gen == g) {
                if (global_ns() - t0 > 2000000000ull) {
                    atomicOr(err, ERR_BARRIER);
                    s_ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

// The barrier alone, for its self-test: every CTA passes `rounds` barriers
// that expect `expect` arrivals.
__global__ void k_barrier_selftest(GridBarrier *bar, unsigned expect, int rounds, unsigned long long *err,
                                   unsigned *passed) {
    for (int r = 0; r < rounds; ++r) {
        if (!grid_barrier(bar, expect, err)) return;
        if (threadIdx.x == 0) atomicAdd(passed, 1u);
    }
}

template <int TPL, typename CT>
__global__ void __launch_bounds__(kPersistThreads, PULDA_PERSIST_MINB) k_batch_sweep_persistent(BatchLaunch b) {
    extern __shared__ uint32_t psm[];
    __shared__ int scan_tmp[kPersistThreads / 32 + 1];
    __shared__ int s_item;
    __shared__ uint32_t geo[kGeoLen];
    __shared__ u64 red[kPersistThreads / 32];
    __shared__ u64 s_sum;
    __shared__ int64_t part[kPersistThreads];
    const unsigned nb = gridDim.x;
    unsigned long long *err = b.phi[0].stats + ST_ERROR;
    // counters of the sweep
    if (blockIdx.x == 0) batch_begin_sweep(b.phi, b.n_chains, b.sweep, b.work);
    if (!grid_barrier(b.bar, nb, err)) return;
    // histograms of the most frequent words, chunk by chunk
    for (int c = blockIdx.x; c < b.n_heavy; c += nb) heavy_chunk(b.phi, b.heavy[c], psm);
    if (!grid_barrier(b.bar, nb, err)) return;
    // counts and Poisson draws, (chain, word) items most frequent first
    {
        int geo_chain = -1;
        for (;;) {
            if (threadIdx.x == 0) s_item = atomicAdd(&b.work[0], 1);
            __syncthreads();
            const int item = s_item;
            __syncthreads();
            if (item >= b.n_phi_items) break;
            const int2 it = b.phi_items[item];
            if (it.x != geo_chain) {
                for (int i = threadIdx.x; i < kGeoLen; i += kPersistThreads) geo[i] = b.phi[it.x].tab.geo[i];
                geo_chain = it.x;
                __syncthreads();
            }
            phi_word<kPersistThreads>(b.phi[it.x], it.y, true, psm, psm + b.kmax, scan_tmp, geo);
        }
    }
    if (!grid_barrier(b.bar, nb, err)) return;
    // rows whose draws summed to zero, one CTA per chain
    for (int c = blockIdx.x; c < b.n_chains; c += nb) phi_fixup_chain<kPersistThreads>(b.phi[c], red, &s_sum);
    if (!grid_barrier(b.bar, nb, err)) return;
    for (int c = blockIdx.x; c < b.n_chains; c += nb) colptr_chain(b.phi[c], part);
    if (!grid_barrier(b.bar, nb, err)) return;
    // per-word tables, one warp per (chain, word)
    {
        const int wid = static_cast<int>(blockIdx.x) * kPersistWarps + (threadIdx.x >> 5);
        const int nw = static_cast<int>(nb) * kPersistWarps;
        for (int i = wid; i < b.n_phi_items; i += nw) {
            const int2 it = b.phi_items[i];
            phi_tables_word_warp(b.phi[it.x], it.y);
        }
    }
    if (!grid_barrier(b.bar, nb, err)) return;
    // z-step, one warp per (chain, document), longest first
    {
        const int lane = threadIdx.x & 31;
        uint32_t *m = psm + static_cast<size_t>(threadIdx.x >> 5) * z_warp_words_t<CT>(b.kmax);
        u64 *wcnt = z_warp_counters_t<CT>(m, b.kmax);
        zero_warp_counters(wcnt);
        for (;;) {
            int item = 0;
            if (lane == 0) item = atomicAdd(&b.work[1], 1);
            item = __shfl_sync(0xFFFFFFFFu, item, 0);
            if (item >= b.n_z_items) break;
            const int2 it = b.z_items[item];
            const ZArgs &a = b.z[it.x];
            const int64_t s0 = a.doc_off[it.y];
            DocRun r{a.w + s0, a.z + s0, static_cast<int>(a.doc_off[it.y + 1] - s0), a.seed, a.index_base + s0,
                     sweep_of(a), 0, a.doc_off[it.y + 1] - s0, 1};
            z_doc_warp_t<TPL, CT>(a, m, r, wcnt, nullptr);
            flush_warp_counters(a.stats, wcnt);
        }
    }
}

cudaError_t launch_barrier_selftest(GridBarrier *bar, int blocks, int missing, int rounds, unsigned long long *err,
                                    unsigned *passed, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(32);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_barrier_selftest, bar, static_cast<unsigned>(blocks + missing), rounds, err,
                              passed);
}

size_t batch_persistent_smem(int kmax, bool narrow) {
    return std::max({phi_counts_smem(kmax), sizeof(uint32_t) * static_cast<size_t>(kmax),
                     z_step_smem(kmax, kPersistWarps, narrow)});
}

using PersistKernel = void (*)(BatchLaunch);
static PersistKernel persistent_kernel(int kmax, bool narrow) {
    switch (z_lane_topics(kmax)) {
        case 8: return narrow ? k_batch_sweep_persistent<8, uint16_t> : k_batch_sweep_persistent<8, uint32_t>;
        case 16: return narrow ? k_batch_sweep_persistent<16, uint16_t> : k_batch_sweep_persistent<16, uint32_t>;
        case 32: return narrow ? k_batch_sweep_persistent<32, uint16_t> : k_batch_sweep_persistent<32, uint32_t>;
        default: return narrow ? k_batch_sweep_persistent<64, uint16_t> : k_batch_sweep_persistent<64, uint32_t>;
    }
}

int batch_persistent_blocks_per_sm(int kmax, bool narrow) {
    PersistKernel kern = persistent_kernel(kmax, narrow);
    allow_dynamic_smem(kern);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kPersistThreads, batch_persistent_smem(kmax, narrow));
    return n;
}

cudaError_t launch_batch_sweep_persistent(const BatchLaunch &b, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(b.persist_grid));
    cfg.blockDim = dim3(kPersistThreads);
    cfg.dynamicSmemBytes = batch_persistent_smem(b.kmax, b.narrow != 0);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, persistent_kernel(b.kmax, b.narrow != 0), b);
}

int batch_phi_blocks_per_sm(int kmax) {
    allow_dynamic_smem(k_phi_counts_multi);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_phi_counts_multi, kPhiBlock, phi_counts_smem(kmax));
    return n > 0 ? n : 1;
}

int batch_z_blocks_per_sm(int kmax, int warps, bool narrow) {
    ZMultiKernel kern = z_multi_kernel(kmax, narrow);
    allow_dynamic_smem(kern);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * warps, z_step_smem(kmax, warps, narrow));
    return n > 0 ? n : 1;
}

using ServeKernel = void (*)(ZArgs, ServeSlot *, const int32_t *, int, const int32_t *, int16_t *, int64_t, int *,
                            uint64_t);
static ServeKernel serve_kernel(int K, bool narrow) {
    switch (z_lane_topics(K)) {
        case 8: return narrow ? k_serve_step<8, uint16_t> : k_serve_step<8, uint32_t>;
        case 16: return narrow ? k_serve_step<16, uint16_t> : k_serve_step<16, uint32_t>;
        case 32: return narrow ? k_serve_step<32, uint16_t> : k_serve_step<32, uint32_t>;
        default: return narrow ? k_serve_step<64, uint16_t> : k_serve_step<64, uint32_t>;
    }
}

void launch_serve_step(const ZArgs &a, ServeSlot *slots, const int32_t *active, int n_active, const int32_t *arena_w,
                       int16_t *arena_z, int64_t slice, int *work, int warps_per_block, int grid, uint64_t window_ns,
                       bool narrow, cudaStream_t st) {
    if (n_active <= 0) return;
    cudaMemsetAsync(work, 0, sizeof(int), st);
    const int need = (n_active + warps_per_block - 1) / warps_per_block;
    ServeKernel kern = serve_kernel(a.K, narrow);
    kern<<<std::min(grid, need), 32 * warps_per_block, z_step_smem(a.K, warps_per_block, narrow), st>>>(
        a, slots, active, n_active, arena_w, arena_z, slice, work, window_ns);
}

int serve_blocks_per_sm(int K, int warps_per_block) {
    // the 32-bit instantiation: its shared memory bounds the 16-bit one's
    for (bool narrow : {true, false}) allow_dynamic_smem(serve_kernel(K, narrow));
    ServeKernel kern = serve_kernel(K, false);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * warps_per_block, z_step_smem(K, warps_per_block));
    return n > 0 ? n : 1;
}

void launch_doc_topic(const int64_t *doc_off, int64_t D, const int16_t *z, int K, int32_t *m_dk, cudaStream_t st) {
    if (D <= 0) return;
    cudaMemsetAsync(m_dk, 0, sizeof(int32_t) * static_cast<size_t>(D) * K, st);
    const int grid = static_cast<int>(std::min<int64_t>((D * 32 + 255) / 256, 8LL * sm_count() * 8));
    k_doc_topic<<<grid, 256, 0, st>>>(doc_off, D, z, K, m_dk);
}

void launch_n_dense(const PhiArgs &a, int32_t *n_kv, cudaStream_t st) {
    cudaMemsetAsync(n_kv, 0, sizeof(int32_t) * static_cast<size_t>(a.K) * a.V, st);
    k_n_dense<<<(a.V + 255) / 256, 256, 0, st>>>(a, n_kv);
}

void launch_phi_values(const PhiArgs &a, float *phi, cudaStream_t st) {
    k_phi_values<<<4 * sm_count(), 256, 0, st>>>(a, phi);
}

}  // namespace pulda
