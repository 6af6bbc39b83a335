// The grouped z-step: four documents per warp, eight lanes per document.
//
// What a token costs on the one-warp kernel (kernels.cu) is mostly work that
// does not grow with its intersection: reading its staged record, removing
// and adding back its topic, the scan of the lanes' partial sums, the draw and
// the search.  Here the 32 lanes of a warp carry four documents, eight lanes
// each, so each of those instructions serves four tokens at once; the
// intersection itself (the only part that grows with K_d and K_v) costs the
// same per token as before.  Draws, sums and their topic order are those of
// Algorithm 2's z-step ("Efficient sampling of z", Eqs. 10-11) in the exact
// integer arithmetic of the one-warp kernel, so every topic and every counter
// is identical.
//
// Lane j of document slot g owns the TL = 32 WPL consecutive topics
// [TL j, TL j + TL) of its document: their counts m (uint16, in a shared
// memory region only that lane touches while tokens are drawn, so the count
// updates need no warp barrier), the matching WPL words of the document's
// nonzero-topic bitmap (registers) and of the token's word's bitmap row (one
// aligned load, fetched a token ahead).  Per token each lane sums q_{k,v} m_k
// over its part of the intersection, reading q from the word's dense row; an
// 8-lane scan gives the prefix in ascending topic order, the draw
// r = floor(u (A + 2^16 B)) takes the alias table when r < A, else the lane
// whose prefix passes (r - A) / 2^16 walks its bits to the topic.
//
// Requires K <= kMaxKGrouped, a dense q row for every word, and documents of at
// most kMaxGroupDocLen tokens (uint16 counts); the host routes anything else to
// the one-warp and cooperative kernels.
#include <algorithm>
#include <cstdint>

#include "device_rng.cuh"
#include "pulda_internal.h"
#include "zstep.cuh"
#include "checks.cuh"

namespace pulda {
namespace {

constexpr int kGLanes = 8;                 // lanes per document
constexpr int kGDocs = 32 / kGLanes;       // documents per warp
#ifndef PULDA_ZG_WARPS
#define PULDA_ZG_WARPS 2
#endif
constexpr int kGWarps = PULDA_ZG_WARPS;    // warps per CTA
#ifndef PULDA_ZG_MINB
#define PULDA_ZG_MINB 8
#endif
// A lane's q loads of one token are asynchronous copies into its own stage
// of this many shared-memory slots, all in flight at once, then one wait: a
// token costs one round trip to L2 instead of one per intersection element.
// A lane with more elements takes them in several rounds.
#ifndef PULDA_ZG_STAGE
#define PULDA_ZG_STAGE 8
#endif
constexpr int kGStage = PULDA_ZG_STAGE;
// Each of a lane's words first takes up to this many intersection elements
// into registers, the loads of all words issued before any is used; only
// the elements beyond them go through the stage.
#ifndef PULDA_ZG_SLOTS
#define PULDA_ZG_SLOTS 6
#endif
constexpr int kGSlots = PULDA_ZG_SLOTS;

// Shared memory of one warp, in 32-bit words: 32 lane regions of
// (TL + 2) uint16 counts (the extra word skews the regions over the banks),
// the staged records of 8 tokens per document (two uint4 each), the warp's
// six 64-bit counters, then the lanes' q stages (slot u of lane l at
// 32 u + l) and the topics they hold (bytes, same order).
__host__ __device__ constexpr int zg_region_words(int wpl) { return 16 * wpl + 1; }
__host__ __device__ constexpr int zg_stage_off(int wpl) { return 32 * zg_region_words(wpl) + kGDocs * kGLanes * 8 + 12; }
__host__ __device__ constexpr int zg_warp_words(int wpl) { return zg_stage_off(wpl) + 32 * kGStage + 8 * kGStage; }
// the records start 16-byte aligned, the counters 8-byte aligned, and so does
// every warp's area
static_assert((32 * zg_region_words(1)) % 4 == 0 && (32 * zg_region_words(2)) % 4 == 0 &&
              (32 * zg_region_words(4)) % 4 == 0, "records must start 16-byte aligned");
static_assert(zg_warp_words(1) % 4 == 0 && zg_warp_words(2) % 4 == 0 && zg_warp_words(4) % 4 == 0,
              "warp areas must start 16-byte aligned");

// Loads a lane's WPL consecutive words of a bitmap row (aligned: rows are
// multiples of 8 WPL words and a lane starts at WPL j).
template <int WPL>
__device__ __forceinline__ void load_bits(const uint32_t *p, uint32_t (&b)[WPL]) {
    if constexpr (WPL == 4) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
    } else if constexpr (WPL == 2) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        b[0] = v.x; b[1] = v.y;
    } else {
        b[0] = __ldg(p);
    }
}

// Stages token i (global index gi) of a document:
//   rec[0] = {Philox x0, x1, sigma_a lo, hi}
//   rec[1] = {offset of its word's dense q row, offset of its word's bitmap row, K_v | old topic << 16,
//             alias-table outcome}
// and returns its current topic.
__device__ __forceinline__ int zg_stage(const ZArgs &a, uint32_t sweep, int64_t gi, uint4 *rec) {
    const int wv = a.w[gi];
    const int zo = guard_index(a.z[gi], a.K, a.stats);
    const uint64_t t = static_cast<uint64_t>(a.index_base + gi);
    const U4 x = draw(a.seed, static_cast<uint32_t>(t), static_cast<uint32_t>(t >> 32), sweep, TAG_Z, 0);
    const int64_t cb = a.col_ptr[wv];
    const int nw = static_cast<int>(a.col_ptr[wv + 1] - cb);
    const u64 Av = a.A[wv];
    int ta = 0;
    if (nw > 0) {
        const uint32_t sl = __umulhi(x.z, static_cast<uint32_t>(nw));
        ta = alias_outcome(a, cb + sl, x.w);
    }
    int ds = a.dense_slot[wv];
    if (ds < 0) {                 // the host sends only corpora whose every word has a row
        atomicOr(&a.stats[ST_ERROR], ERR_INTERNAL);
        ds = 0;
    }
    const uint32_t qoff = static_cast<uint32_t>(ds) * static_cast<uint32_t>(a.K);
    rec[0] = make_uint4(x.x, x.y, static_cast<uint32_t>(Av), static_cast<uint32_t>(Av >> 32));
    rec[1] = make_uint4(qoff, static_cast<uint32_t>(wv) * static_cast<uint32_t>(a.KWp),
                        static_cast<uint32_t>(nw) | (static_cast<uint32_t>(zo) << 16), static_cast<uint32_t>(ta));
    return zo;
}

// A 4-byte asynchronous copy from global to this thread's shared memory, and
// the wait for every copy this thread has issued.
__device__ __forceinline__ void cp_async4(uint32_t *smem, const uint32_t *gmem) {
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <int WPL>
__global__ void __launch_bounds__(32 * kGWarps, PULDA_ZG_MINB) k_z_step_grouped(ZArgs a) {
    constexpr int TL = 32 * WPL;                 // topics per lane
    constexpr int RW = 16 * WPL + 1;             // 32-bit words per lane region
    extern __shared__ uint32_t zg_sm[];
    const int lane = threadIdx.x & 31;
    const int g = lane >> 3, gl = lane & 7;
    const unsigned gmask = 0xFFu << (8 * g);
    const int K = a.K;
    uint32_t *wsm = zg_sm + static_cast<size_t>(threadIdx.x >> 5) * zg_warp_words(WPL);
    uint32_t *myw = wsm + lane * RW;                                  // this lane's counts, as uint16 pairs
    uint16_t *my = reinterpret_cast<uint16_t *>(myw);
    uint4 *rec = reinterpret_cast<uint4 *>(wsm + 32 * RW);
    u64 *wcnt = reinterpret_cast<u64 *>(rec + 2 * kGDocs * kGLanes);
    uint32_t *stq = wsm + zg_stage_off(WPL) + lane;                   // q stage, slot u at stq[32 u]
    uint8_t *stk = reinterpret_cast<uint8_t *>(wsm + zg_stage_off(WPL) + 32 * kGStage) + lane;   // its topics
    zero_warp_counters(wcnt);
    const uint32_t sweep = sweep_of(a);
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.work, 1);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (static_cast<int64_t>(item) * kGDocs >= a.D) break;
        const int64_t di = static_cast<int64_t>(item) * kGDocs + g;
        int64_t s = 0;
        int len = 0;
        if (di < a.D) {
            const int d = a.doc_order[di];
            s = a.doc_off[d];
            len = static_cast<int>(a.doc_off[d + 1] - s);
        }
        // m_d from the document's current topics: each count goes to its
        // owner's region
        for (int t = 0; t < RW; ++t) myw[t] = 0u;
        __syncwarp();
        for (int i = gl; i < len; i += kGLanes) {
            const int k = guard_index(a.z[s + i], K, a.stats);
            const int j = k / TL, t = k - j * TL;
            atomicAdd(&wsm[(8 * g + j) * RW + (t >> 1)], 1u << (16 * (t & 1)));
        }
        __syncwarp();
        // this lane's bits of m_d's nonzero topics, and K_d
        uint32_t mb[WPL];
#pragma unroll
        for (int w = 0; w < WPL; ++w) {
            uint32_t bb = 0;
#pragma unroll 4
            for (int p = 0; p < 16; ++p) {
                const uint32_t pr = myw[16 * w + p];
                bb |= ((pr & 0xFFFFu) ? 1u : 0u) << (2 * p);
                bb |= ((pr >> 16) ? 1u : 0u) << (2 * p + 1);
            }
            mb[w] = bb;
        }
        int kd = 0;
#pragma unroll
        for (int w = 0; w < WPL; ++w) kd += __popc(mb[w]);
        kd += __shfl_xor_sync(0xFFFFFFFFu, kd, 1);
        kd += __shfl_xor_sync(0xFFFFFFFFu, kd, 2);
        kd += __shfl_xor_sync(0xFFFFFFFFu, kd, 4);
        const int maxlen = __reduce_max_sync(0xFFFFFFFFu, static_cast<unsigned>(len));
        for (int t0 = 0; t0 < maxlen; t0 += kGLanes) {
            const int cnt = max(0, min(kGLanes, len - t0));             // this document's tokens in the block
            const int maxcnt = static_cast<int>(__reduce_max_sync(0xFFFFFFFFu, static_cast<unsigned>(cnt)));
            uint4 *grec = rec + 2 * kGLanes * g;
            int znew = 0;
            if (gl < cnt) znew = zg_stage(a, sweep, s + t0 + gl, grec + 2 * gl);
            __syncwarp();
            uint32_t bn[WPL];
#pragma unroll
            for (int w = 0; w < WPL; ++w) bn[w] = 0u;
            if (cnt > 0) load_bits<WPL>(a.bits + grec[1].y + WPL * gl, bn);
            // this block's counters: c_min = sum of min(K_d, K_v) (the same in
            // the document's 8 lanes); c_cnt = tokens with K_d < K_v (bits
            // 0-5), alias draws (6-11), zero-mass tokens (12-17), this lane's
            // share of |J| (from 18)
            uint32_t c_min = 0, c_cnt = 0;
            for (int tt = 0; tt < maxcnt; ++tt) {
                const bool act = tt < cnt;
                const uint4 r0 = grec[2 * tt], r1 = grec[2 * tt + 1];
                const int kold = static_cast<int>(r1.z >> 16);
                const int n_w = static_cast<int>(r1.z & 0xFFFFu);
                const u64 At = (static_cast<u64>(r0.w) << 32) | r0.z;
                const u64 U = (static_cast<u64>(r0.x) << 32) | r0.y;
                uint32_t bw[WPL];
#pragma unroll
                for (int w = 0; w < WPL; ++w) bw[w] = bn[w];
                if (tt + 1 < cnt) load_bits<WPL>(a.bits + grec[2 * tt + 3].y + WPL * gl, bn);
                // remove token i: m^{-i} (by the lane that owns its topic)
                bool gone = false;
                if (act && (kold / TL) == gl) {
                    const int t = kold - gl * TL;
                    const uint32_t o = my[t];
                    my[t] = static_cast<uint16_t>(o - 1u);
                    if (o == 1u) {
                        gone = true;
                        // a select per word, so mb stays in registers
#pragma unroll
                        for (int w = 0; w < WPL; ++w) mb[w] &= (t >> 5) == w ? ~(1u << (t & 31)) : 0xFFFFFFFFu;
                    }
                }
                if (__ballot_sync(0xFFFFFFFFu, gone) & gmask) --kd;
                if (act) {
                    c_min += static_cast<uint32_t>(kd < n_w ? kd : n_w);
                    c_cnt += kd < n_w ? 1u : 0u;
                }
                // this lane's part of the intersection (ascending topics) and its
                // sum of q m: the q loads of up to kGStage elements are copies in
                // flight together
                const uint32_t *qrow = a.qdense + r1.x + gl * TL;
                uint32_t rem[WPL];
                int jc = 0;
#pragma unroll
                for (int w = 0; w < WPL; ++w) {
                    rem[w] = act ? (bw[w] & mb[w]) : 0u;
                    jc += __popc(rem[w]);
                }
                c_cnt += static_cast<uint32_t>(jc) << 18;
                // registers: the first kGSlots elements of every word, their loads
                // issued together; stage: the rest (n of them, ascending)
                uint32_t qv[WPL][kGSlots];
                int bp[WPL][kGSlots];
                uint32_t rr[WPL];
#pragma unroll
                for (int w = 0; w < WPL; ++w) {
                    rr[w] = rem[w];
#pragma unroll
                    for (int u = 0; u < kGSlots; ++u) {
                        bp[w][u] = -1;
                        qv[w][u] = 0u;
                        if (rr[w]) {
                            const int b = __ffs(rr[w]) - 1;
                            rr[w] &= rr[w] - 1u;
                            bp[w][u] = b;
                            qv[w][u] = __ldg(qrow + 32 * w + b);
                        }
                    }
                }
                int n = 0;
                bool spill = false;          // more leftovers than the stage holds
#pragma unroll
                for (int w = 0; w < WPL; ++w) {
                    for (uint32_t bb = rr[w]; bb; bb &= bb - 1u) {
                        const int k = 32 * w + __ffs(bb) - 1;
                        if (n < kGStage) {
                            cp_async4(stq + 32 * n, qrow + k);
                            stk[32 * n] = static_cast<uint8_t>(k);
                            ++n;
                        } else {
                            spill = true;
                        }
                    }
                }
                u64 sw[WPL];
#pragma unroll
                for (int w = 0; w < WPL; ++w) {
                    u64 t = 0;
#pragma unroll
                    for (int u = 0; u < kGSlots; ++u)
                        if (bp[w][u] >= 0) t += static_cast<u64>(qv[w][u]) * my[32 * w + bp[w][u]];
                    sw[w] = t;
                }
                cp_async_wait_all();
                for (int u = 0; u < n; ++u) {
                    const int k = stk[32 * u];
                    const u64 p = static_cast<u64>(stq[32 * u]) * my[k];
#pragma unroll
                    for (int w = 0; w < WPL; ++w) sw[w] += (k >> 5) == w ? p : 0ull;
                }
                if (spill) {                 // past the stage: one at a time
                    int seen = 0;
#pragma unroll
                    for (int w = 0; w < WPL; ++w) {
                        for (uint32_t bb = rr[w]; bb; bb &= bb - 1u) {
                            const int k = 32 * w + __ffs(bb) - 1;
                            if (seen++ >= kGStage) sw[w] += static_cast<u64>(__ldg(qrow + k)) * my[k];
                        }
                    }
                }
                u64 acc = 0;
#pragma unroll
                for (int w = 0; w < WPL; ++w) acc += sw[w];
                // inclusive scan over the document's 8 lanes (ascending topics)
                u64 incl = acc;
#pragma unroll
                for (int o = 1; o < kGLanes; o <<= 1) {
                    const u64 y = __shfl_up_sync(0xFFFFFFFFu, incl, o, kGLanes);
                    if (gl >= o) incl += y;
                }
                const u64 B = __shfl_sync(0xFFFFFFFFu, incl, 8 * g + 7);
                const u64 T = At + (B << kFracBits);
                int knew = kold;
                bool need = false;
                u64 rb = 0;
                if (act) {
                    if (T == 0) {
                        c_cnt += 1u << 12;
                    } else {
                        const u64 r = __umul64hi(U, T);
                        if (r < At) {
                            knew = static_cast<int>(r1.w);
                            c_cnt += 1u << 6;
                        } else {
                            need = true;
                            rb = (r - At) >> kFracBits;
                        }
                    }
                }
                const uint32_t gb = (__ballot_sync(0xFFFFFFFFu, need && rb < incl) & gmask) >> (8 * g);
                const int L = gb ? __ffs(gb) - 1 : 0;
                int f = -1;
                if (need && gb && gl == L) {
                    // the first word whose running sum passes rb, then its elements
                    // in ascending order (q re-read: it was just fetched)
                    u64 run = incl - acc;
                    uint32_t wbits = 0;
                    int wbase = 0;
                    bool sel = false;
#pragma unroll
                    for (int w = 0; w < WPL; ++w) {
                        if (!sel) {
                            if (w == WPL - 1 || rb < run + sw[w]) {
                                wbits = rem[w];
                                wbase = 32 * w;
                                sel = true;
                            } else {
                                run += sw[w];
                            }
                        }
                    }
                    for (uint32_t bb = wbits; bb; bb &= bb - 1u) {
                        const int b = __ffs(bb) - 1;
                        run += static_cast<u64>(__ldg(qrow + wbase + b)) * my[wbase + b];
                        if (rb < run) { f = gl * TL + wbase + b; break; }
                    }
                }
                const int found = __shfl_sync(0xFFFFFFFFu, f, 8 * g + L);
                if (need) {
                    if (found < 0) {
                        if (gl == 0) atomicOr(&a.stats[ST_ERROR], ERR_INTERNAL);
                    } else {
                        knew = found;
                    }
                }
                // add token i back with its new topic (by the lane that owns it)
                if (act) knew = guard_index(knew, K, a.stats);
                bool born = false;
                if (act && (knew / TL) == gl) {
                    const int t = knew - gl * TL;
                    const uint32_t o = my[t];
                    my[t] = static_cast<uint16_t>(o + 1u);
                    if (o == 0u) {
                        born = true;
#pragma unroll
                        for (int w = 0; w < WPL; ++w) mb[w] |= (t >> 5) == w ? 1u << (t & 31) : 0u;
                    }
                }
                if (__ballot_sync(0xFFFFFFFFu, born) & gmask) ++kd;
                if (gl == tt) znew = knew;
            }
            if (gl < cnt) a.z[s + t0 + gl] = static_cast<int16_t>(znew);
            {   // the block's counts into the warp's 64-bit counters, lane j its counter j;
                // a document's counts are the same in its 8 lanes: take lane 0's
                const bool g0 = gl == 0;
                const uint32_t ntok = __reduce_add_sync(0xFFFFFFFFu, g0 ? static_cast<uint32_t>(cnt) : 0u);
                const uint32_t nab = __reduce_add_sync(0xFFFFFFFFu, g0 ? (c_cnt >> 6) & 63u : 0u);
                const uint32_t nmin = __reduce_add_sync(0xFFFFFFFFu, g0 ? c_min : 0u);
                const uint32_t nzero = __reduce_add_sync(0xFFFFFFFFu, g0 ? (c_cnt >> 12) & 63u : 0u);
                const uint32_t nj = __reduce_add_sync(0xFFFFFFFFu, c_cnt >> 18);
                const uint32_t ndoc = __reduce_add_sync(0xFFFFFFFFu, g0 ? c_cnt & 63u : 0u);
                const uint32_t v = lane == 0 ? ntok : lane == 1 ? nab : lane == 2 ? nmin
                                 : lane == 3 ? nzero : lane == 4 ? nj : ndoc;
                if (lane < 6) wcnt[lane] += v;
            }
            __syncwarp();     // every lane is done with the records before they are restaged
        }
    }
    flush_warp_counters(a.stats, wcnt);
}

template <int WPL>
size_t zg_smem() { return sizeof(uint32_t) * static_cast<size_t>(zg_warp_words(WPL)) * kGWarps; }

template <int WPL>
int zg_blocks_per_sm() {
    allow_dynamic_smem(k_z_step_grouped<WPL>);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_z_step_grouped<WPL>, 32 * kGWarps, zg_smem<WPL>());
    return b > 0 ? b : 1;
}

template <int WPL>
void zg_launch(const ZArgs &a, int grid, cudaStream_t st) {
    k_z_step_grouped<WPL><<<grid, 32 * kGWarps, zg_smem<WPL>(), st>>>(a);
}

}  // namespace

int z_groups_blocks_per_sm(int K) {
    const int wpl = bitmap_row_words(K) / 8;
    return wpl == 1 ? zg_blocks_per_sm<1>() : wpl == 2 ? zg_blocks_per_sm<2>() : zg_blocks_per_sm<4>();
}

void launch_z_step_groups(const ZArgs &a, int grid, cudaStream_t st) {
    if (a.D <= 0) return;
    const int wpl = a.KWp / 8;
    if (wpl == 1) zg_launch<1>(a, grid, st);
    else if (wpl == 2) zg_launch<2>(a, grid, st);
    else zg_launch<4>(a, grid, st);
}

}  // namespace pulda
