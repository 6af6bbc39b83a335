// The cooperative z-step: one CTA per long document (corpus, fold-in, serving
// and batched forms).  Same draws, in the same order, as the one-warp kernel
// of kernels.cu, so the topics are identical.
#include <algorithm>
#include <cstdint>

#include "device_rng.cuh"
#include "pulda_internal.h"
#include "zstep.cuh"
#include "checks.cuh"

namespace pulda {
namespace {

// ============================================================== cooperative z-step
// A document's tokens are strictly sequential, so on one warp the longest
// documents outlast the rest of the z-step: a few microseconds per token
// (every token waits on its q gathers, its scan and its draw in turn) times
// thousands of tokens, while the other warps have long finished.  Here the
// kCoopWarps warps of a CTA share one document, token by token.  The token's
// intersection is split over the CTA's kCoopSlots lanes ("slots") in
// ascending topic order: on the document side slot g owns the R consecutive
// topics [g R, g R + R) (R the smallest power of two with 32 KW <= R slots),
// on the column side a contiguous segment of the word's column.  Each slot
// gathers its few q values at once, every warp scans its slots, the warps'
// totals meet in shared memory (barrier A), and the slot whose prefix passes
// the draw reads off the topic, updates m and publishes it (barrier B).  The
// sums are the same exact integers in the same topic order as the one-warp
// kernel's, so every draw, and every topic, is identical.
#ifndef PULDA_COOP_WARPS
#define PULDA_COOP_WARPS 4
#endif
constexpr int kCoopWarps = PULDA_COOP_WARPS;
constexpr int kCoopSlots = 32 * kCoopWarps;
#ifndef PULDA_COOP_GATHER
#define PULDA_COOP_GATHER 3
#endif
constexpr int kCoopGather = PULDA_COOP_GATHER;   // document-side q loads issued together per slot
// 64 registers, as the one-warp kernel (8 CTAs of four warps per SM); the
// serving form needs 72 (7 CTAs of four warps).
constexpr int kCoopMinBlocks = 32 / kCoopWarps;
constexpr int kCoopServeMinBlocks = 28 / kCoopWarps > 0 ? 28 / kCoopWarps : 1;

struct CoopXch {
    u64 tot[kCoopWarps];    // each warp's sum of q m over its slots (this token)
    int kdp[kCoopWarps];    // each warp's share of K_d when the document starts
    int item;               // the document the CTA takes next
    int go;                 // thread 0's reading of the deadline for the next block
    int knew;               // this token's new topic
    uint32_t mkn;           // m^{-i} of the new topic, before the token is added back
};
// Shared memory of a cooperative CTA, in 32-bit words: m_d, the records of
// 32 tokens, the exchange area.
__host__ __device__ __forceinline__ int z_coop_words(int K) {
    return z_m_words(K) + 32 * kTokRecWords + static_cast<int>((sizeof(CoopXch) + 15) / 16) * 4;
}

__device__ void z_doc_coop(const ZArgs &a, uint32_t *sm, DocRun &r, ZCount &st) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = a.K;
    // topic k's count at m[mi(k)], with a zero word before each 32-topic
    // word's counts (sm[0] before word 0, the gap word of word w - 1 before
    // word w): a gather slot past a slot's last bit reads a zero there
    uint32_t *m = sm + 1;
    uint4 *rec = reinterpret_cast<uint4 *>(sm + z_m_words(K));
    uint32_t *drow_of = reinterpret_cast<uint32_t *>(rec + 64);
    CoopXch &x = *reinterpret_cast<CoopXch *>(drow_of + 32);
    const bool use_bm = a.bits != nullptr && a.path != 1;
    int R = 1;
    while (32 * a.KW > R * kCoopSlots) R <<= 1;
    const bool own = use_bm && tid < 32 * a.KW / R;      // this slot owns topics on the document side
    const int wi = own ? (tid * R) >> 5 : 0;              // its bitmap word
    const int sh = (tid * R) & 31;
    const uint32_t mask = own ? (R >= 32 ? 0xFFFFFFFFu : ((1u << R) - 1u) << sh) : 0u;
    if (r.len == 0 || r.budget <= 0) return;
    for (int k = tid; k < K; k += kCoopSlots) m[mi(k)] = 0;
    if (tid == 0) sm[0] = 0;
    for (int w = tid; w + 1 < a.KW; w += kCoopSlots) m[33 * w + 32] = 0;
    __syncthreads();
    for (int i = tid; i < r.len; i += kCoopSlots) atomicAdd(&m[mi(guard_index(r.z[i], K, a.stats))], 1u);
    __syncthreads();
    uint32_t mb = 0;        // this slot's bits of m_d's nonzero topics
    int c = 0;
    if (use_bm) {
        for (int t = 0; t < R && own; ++t) {
            const int k = wi * 32 + sh + t;
            if (k < K && m[mi(k)] > 0) mb |= 1u << (sh + t);
        }
        c = __popc(mb);
    } else {
        for (int k = tid; k < K; k += kCoopSlots) c += m[mi(k)] > 0 ? 1 : 0;
    }
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if (lane == 0) x.kdp[warp] = c;
    __syncthreads();
    int kd = 0;
#pragma unroll
    for (int j = 0; j < kCoopWarps; ++j) kd += x.kdp[j];
    const uint32_t *bits = a.bits;
    const uint32_t sweep_end = r.sweep + static_cast<uint32_t>(r.max_pass_end);
    bool first = true;
    while (r.budget > 0 && r.sweep != sweep_end) {
        const int i0 = r.pos;
        const int cnt = static_cast<int>(min(static_cast<int64_t>(32), min(static_cast<int64_t>(r.len - i0), r.budget)));
        if (tid == 0) x.go = r.deadline == ~0ull || first || global_ns() < r.deadline;
        if (warp == 0 && lane < cnt) stage_token(a, r, i0 + lane, rec + 2 * lane, drow_of + lane);
        __syncthreads();
        if (!x.go) break;     // the same value in every thread: read before any thread can write it again
        first = false;
        uint32_t bm_next = own ? bits[static_cast<int64_t>(rec[1].z) * a.KWp + wi] & mask : 0u;
        for (int tt = 0; tt < cnt; ++tt) {
            const uint4 t0 = rec[2 * tt], t1 = rec[2 * tt + 1];
            const int kold = static_cast<int>(t1.w >> 16);
            const int64_t col = static_cast<int64_t>((static_cast<u64>(t0.y & 0xFFFFu) << 32) | t0.x);
            const int n_w = static_cast<int>(t1.w & 0xFFFFu);
            const u64 At = (static_cast<u64>(t0.w) << 32) | t0.z;
            const u64 U = (static_cast<u64>(t1.x) << 32) | t1.y;
            const int ka = static_cast<int>(t0.y >> 16);
            const uint32_t bm = bm_next;
            if (own && tt + 1 < cnt) bm_next = bits[static_cast<int64_t>(rec[2 * tt + 3].z) * a.KWp + wi] & mask;
            // m^{-i}: the old topic's count less one, applied as each count is read
            const uint32_t mko = m[mi(kold)];
            const int kdi = kd - (mko == 1u ? 1 : 0);
            if (mko == 1u && own && (kold >> 5) == wi) mb &= ~(1u << (kold & 31));
            if (warp == 0) {
                st.add(2, static_cast<u64>(kdi < n_w ? kdi : n_w));
                st.add(5, kdi < n_w ? 1u : 0u);
            }
            const uint32_t drow = drow_of[tt];
            const bool docside = use_bm && drow != 0xFFFFFFFFu && (a.path == 2 || kdi * kDocRatio < n_w * 16);
            const uint32_t *qrow = a.qdense + drow + 32 * wi;
            u64 acc = 0;
            uint32_t rem = 0;
            int j0 = 0, j1 = 0;
            uint32_t qv[kCoopGather];
            int bp[kCoopGather];
            uint32_t rest = 0;
            if (docside) {
                rem = bm & mb;
                st.inter += static_cast<u64>(__popc(rem));
                // the slot's bits from the highest down; a slot past the last
                // bit gets b = -1, q = 0 (no load) and the zero before the word
                uint32_t bb = rem;
#pragma unroll
                for (int t = 0; t < kCoopGather; ++t) {
                    const int b = msb_or_neg1(bb);
                    bb ^= bit_or_zero(b);
                    bp[t] = b;
                    qv[t] = b >= 0 ? qrow[b] : 0u;
                }
#pragma unroll
                for (int t = 0; t < kCoopGather; ++t) {
                    const int k = 32 * wi + bp[t];
                    acc += static_cast<u64>(qv[t]) * (m[33 * wi + bp[t]] - (k == kold ? 1u : 0u));
                }
                rest = bb;
                for (uint32_t b2 = rest; b2;) {
                    const int b = msb_or_neg1(b2);
                    b2 ^= bit_or_zero(b);
                    const int k = 32 * wi + b;
                    acc += static_cast<u64>(qrow[b]) * (m[33 * wi + b] - (k == kold ? 1u : 0u));
                }
            } else {
                const int seg = (n_w + kCoopSlots - 1) / kCoopSlots;
                j0 = min(seg * tid, n_w);
                j1 = min(j0 + seg, n_w);
                unsigned nj = 0;
#pragma unroll 4
                for (int j = j0; j < j1; ++j) {
                    const int k = guard_index(a.topic[col + j], K, a.stats);
                    const uint32_t mk = m[mi(k)] - (k == kold ? 1u : 0u);
                    acc += static_cast<u64>(a.q[col + j]) * mk;
                    nj += mk != 0u;
                }
                st.inter += static_cast<u64>(nj);
            }
            const u64 incl = warp_incl_scan64(acc);
            if (lane == 31) x.tot[warp] = incl;
            __syncthreads();                                  // A: the warps' totals
            u64 B = 0;
            u64 tot[kCoopWarps];
#pragma unroll
            for (int j = 0; j < kCoopWarps; ++j) {
                tot[j] = x.tot[j];
                B += tot[j];
            }
            const u64 T = At + (B << kFracBits);
            int knew = kold;
            bool upd = tid == 0;        // who updates m and publishes the topic
            if (T == 0) {
                if (warp == 0) st.add(3, 1);
            } else {
                const u64 rr = __umul64hi(U, T);
                if (rr < At) {
                    knew = ka;
                    if (warp == 0) st.add(1, 1);
                } else {
                    const u64 rb = (rr - At) >> kFracBits;   // < B
                    int selw = kCoopWarps;
                    u64 lo = 0;
#pragma unroll
                    for (int j = 0; j < kCoopWarps; ++j) {
                        if (selw == kCoopWarps) {
                            if (rb < lo + tot[j]) selw = j;
                            else lo += tot[j];
                        }
                    }
                    if (selw == kCoopWarps) {
                        if (tid == 0) atomicOr(&a.stats[ST_ERROR], ERR_INTERNAL);
                    } else {
                        upd = false;
                        if (warp == selw) {
                            const u64 rbl = rb - lo;
                            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, rbl < incl);   // lane 31 at least
                            if (lane == (bal ? __ffs(bal) - 1 : 31)) {
                                upd = true;
                                int f = -1;
                                if (docside) {
                                    // down from the slot's inclusive sum: the topic whose
                                    // term takes it to rbl or below
                                    u64 run = incl;
#pragma unroll
                                    for (int t = 0; t < kCoopGather; ++t) {
                                        const int k = 32 * wi + bp[t];
                                        run -= static_cast<u64>(qv[t]) * (m[33 * wi + bp[t]] - (k == kold ? 1u : 0u));
                                        if (rbl >= run) { f = k; break; }
                                    }
                                    for (uint32_t b2 = rest; f < 0 && b2;) {
                                        const int b = msb_or_neg1(b2);
                                        b2 ^= bit_or_zero(b);
                                        const int k = 32 * wi + b;
                                        run -= static_cast<u64>(qrow[b]) * (m[33 * wi + b] - (k == kold ? 1u : 0u));
                                        if (rbl >= run) f = k;
                                    }
                                } else {
                                    u64 run = incl - acc;
                                    for (int j = j0; j < j1; ++j) {
                                        const int k = guard_index(a.topic[col + j], K, a.stats);
                                        run += static_cast<u64>(a.q[col + j]) * (m[mi(k)] - (k == kold ? 1u : 0u));
                                        if (rbl < run) { f = k; break; }
                                    }
                                }
                                if (f < 0) atomicOr(&a.stats[ST_ERROR], ERR_INTERNAL);
                                else knew = f;
                            }
                        }
                    }
                }
            }
            if (upd) {
                knew = guard_index(knew, K, a.stats);
                const uint32_t mkn = knew == kold ? mko - 1u : m[mi(knew)];
                if (knew != kold) {
                    m[mi(kold)] = mko - 1u;
                    m[mi(knew)] = mkn + 1u;
                }
                x.knew = knew;
                x.mkn = mkn;
                r.z[i0 + tt] = static_cast<int16_t>(knew);
            }
            __syncthreads();                                  // B: the new topic, m updated
            const int kn = x.knew;
            const uint32_t mkn = x.mkn;
            kd = kdi + (mkn == 0u ? 1 : 0);
            if (mkn == 0u && own && (kn >> 5) == wi && ((mask >> (kn & 31)) & 1u)) mb |= 1u << (kn & 31);
        }
        if (warp == 0) st.add(0, static_cast<u64>(cnt));
        r.budget -= cnt;
        r.pos += cnt;
        if (r.pos == r.len) { r.pos = 0; r.sweep += 1; }
    }
}

// The longest documents of a pass, one CTA each (dynamically scheduled,
// longest first): doc_order[0 .. n_coop).
__global__ void __launch_bounds__(kCoopSlots, kCoopMinBlocks) k_z_step_coop(ZArgs a, int n_coop, int *work) {
    extern __shared__ uint32_t zsm[];
    CoopXch &x = *reinterpret_cast<CoopXch *>(zsm + z_m_words(a.K) + 32 * kTokRecWords);
    ZCount st;
    const uint32_t sweep = sweep_of(a);
    for (;;) {
        if (threadIdx.x == 0) x.item = atomicAdd(work, 1);
        __syncthreads();
        const int item = x.item;
        __syncthreads();
        if (item >= n_coop) break;
        const int d = a.doc_order[item];
        const int64_t s = a.doc_off[d];
        const int len = static_cast<int>(a.doc_off[d + 1] - s);
        DocRun r{a.w + s, a.z + s, len, a.seed, a.index_base + s, sweep, 0, len, 1};
        z_doc_coop(a, zsm, r, st);
    }
    flush_warp_z_stats(a.stats, st);
}

// Many chains: the longest documents of every chain, one CTA each (the
// cooperative z-step); items[0 .. n_items) are (chain, document) pairs.
__global__ void __launch_bounds__(kCoopSlots, kCoopMinBlocks) k_z_step_coop_multi(const ZArgs *chains,
                                                                                   const int2 *items, int n_items,
                                                                                   int *work, int kmax) {
    extern __shared__ uint32_t zsm[];
    int *item_sh = reinterpret_cast<int *>(zsm + z_coop_words(kmax));    // beyond every chain's layout
    for (;;) {
        if (threadIdx.x == 0) *item_sh = atomicAdd(work, 1);
        __syncthreads();
        const int item = *item_sh;
        __syncthreads();
        if (item >= n_items) break;
        const int2 it = items[item];
        const ZArgs &a = chains[it.x];
        const int64_t s = a.doc_off[it.y];
        const int len = static_cast<int>(a.doc_off[it.y + 1] - s);
        DocRun r{a.w + s, a.z + s, len, a.seed, a.index_base + s, sweep_of(a), 0, len, 1};
        ZCount st;
        z_doc_coop(a, zsm, r, st);
        flush_warp_z_stats(a.stats, st);
    }
}

// The same for the long requests, one CTA of kCoopWarps warps each (the
// cooperative z-step): active[0 .. n_active) are those slots.
__global__ void __launch_bounds__(kCoopSlots, kCoopServeMinBlocks) k_serve_step_coop(ZArgs a, ServeSlot *slots, const int32_t *active,
                                                                     int n_active, const int32_t *arena_w,
                                                                     int16_t *arena_z, int64_t slice, int *work,
                                                                     uint64_t window_ns) {
    extern __shared__ uint32_t zsm[];
    CoopXch &x = *reinterpret_cast<CoopXch *>(zsm + z_m_words(a.K) + 32 * kTokRecWords);
    ZCount st;
    for (;;) {
        __syncthreads();          // every thread has read the previous item and its deadline
        if (threadIdx.x == 0) {
            x.item = atomicAdd(work, 1);
            x.tot[0] = window_ns ? global_ns() + window_ns : ~0ull;
        }
        __syncthreads();
        const int item = x.item;
        const uint64_t deadline = x.tot[0];
        if (item >= n_active) break;
        const int idx = active[item];
        const ServeSlot sl = slots[idx];
        int16_t *z = arena_z + sl.off;
        uint32_t sweep = sl.sweep;
        int pos = sl.pos;
        if (sweep == 0) {
            for (int i = threadIdx.x; i < sl.len; i += kCoopSlots) {
                const U4 u = draw(sl.seed, static_cast<uint32_t>(i), 0u, 0u, TAG_INIT, 0);
                z[i] = static_cast<int16_t>(__umulhi(u.x, static_cast<uint32_t>(a.K)));
            }
            __syncthreads();
            sweep = 1;
            pos = 0;
        }
        DocRun r{arena_w + sl.off, z, sl.len, sl.seed, 0, sweep, pos, slice,
                 static_cast<int>(sl.sweep_end - sweep), deadline};
        z_doc_coop(a, zsm, r, st);
        if (threadIdx.x == 0) {
            slots[idx].sweep = r.sweep;
            slots[idx].pos = r.pos;
        }
    }
    flush_warp_z_stats(a.stats, st);
}

}  // namespace

size_t z_coop_smem(int K) { return sizeof(uint32_t) * static_cast<size_t>(z_coop_words(K)); }

int z_coop_blocks_per_sm(int K) {
    allow_dynamic_smem(k_z_step_coop);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_z_step_coop, kCoopSlots, z_coop_smem(K));
    return b > 0 ? b : 1;
}

void launch_z_step_coop(const ZArgs &a, int n_coop, int *work, int grid, cudaStream_t st) {
    if (n_coop <= 0) return;
    k_z_step_coop<<<std::max(1, std::min(grid, n_coop)), kCoopSlots, z_coop_smem(a.K), st>>>(a, n_coop, work);
}

size_t z_coop_multi_smem(int kmax) { return sizeof(uint32_t) * static_cast<size_t>(z_coop_words(kmax)) + 16; }

int batch_coop_blocks_per_sm(int kmax) {
    allow_dynamic_smem(k_z_step_coop_multi);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_z_step_coop_multi, kCoopSlots, z_coop_multi_smem(kmax));
    return n > 0 ? n : 1;
}

void launch_serve_step_coop(const ZArgs &a, ServeSlot *slots, const int32_t *active, int n_active,
                            const int32_t *arena_w, int16_t *arena_z, int64_t slice, int *work, int grid,
                            uint64_t window_ns, cudaStream_t st) {
    if (n_active <= 0) return;
    cudaMemsetAsync(work, 0, sizeof(int), st);
    k_serve_step_coop<<<std::max(1, std::min(grid, n_active)), kCoopSlots, z_coop_smem(a.K), st>>>(
        a, slots, active, n_active, arena_w, arena_z, slice, work, window_ns);
}

int serve_coop_blocks_per_sm(int K) {
    allow_dynamic_smem(k_serve_step_coop);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_serve_step_coop, kCoopSlots, z_coop_smem(K));
    return n > 0 ? n : 1;
}


void launch_z_step_coop_multi(const ZArgs *chains, const int2 *items, int n_items, int *work, int kmax, int grid,
                              cudaStream_t st) {
    if (n_items <= 0) return;
    k_z_step_coop_multi<<<std::max(1, std::min(grid, n_items)), kCoopSlots, z_coop_multi_smem(kmax), st>>>(
        chains, items, n_items, work, kmax);
}

}  // namespace pulda
