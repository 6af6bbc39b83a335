// What the z-step kernels share (kernels.cu: one warp per document; coop.cu:
// one CTA per document): the per-document run, the staging of a token's
// token-only data, the warp's counters, m_d's shared-memory layout and the
// warp scans.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "device_rng.cuh"
#include "pulda_internal.h"
#include "checks.cuh"

namespace pulda {

typedef unsigned long long u64;

__device__ __forceinline__ u64 warp_sum64(u64 v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ u64 warp_incl_scan64(u64 v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Position of the highest set bit of x, or -1 when x is 0 (PTX bfind).
__device__ __forceinline__ int msb_or_neg1(uint32_t x) {
    int b;
    asm("bfind.u32 %0, %1;" : "=r"(b) : "r"(x));
    return b;
}

// 1 << b for b in [0, 32), 0 for b = -1 (PTX shl clamps the shift at 32).
__device__ __forceinline__ uint32_t bit_or_zero(int b) {
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(1u), "r"(b));
    return r;
}

// The same for a lane's 64 topics (two bitmap words).
__device__ __forceinline__ int msb_or_neg1(uint64_t x) {
    int b;
    asm("bfind.u64 %0, %1;" : "=r"(b) : "l"(x));
    return b;
}
__device__ __forceinline__ uint64_t bit_or_zero64(int b) {
    uint64_t r;
    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(1ull), "r"(b));
    return r;
}

__device__ __forceinline__ uint32_t sweep_of(const ZArgs &a) { return a.sweep_ptr ? *a.sweep_ptr : a.sweep; }

// The document side (for a word with a dense q row) is iterated when
// K_d * kDocRatio < K_v * 16: the paper's "iterate over the smaller" at 16.
// Either side gives the same exact sums; the column side's topic -> m loads
// depend on each other, which makes it the costlier side per element.
#ifndef PULDA_ZDOCRATIO
#define PULDA_ZDOCRATIO 16
#endif

constexpr int kDocRatio = PULDA_ZDOCRATIO;


// m_d is stored skewed, topic k at k + k/32, so the lanes of a warp reading
// topics 32 l + b (lane l, bit b) hit distinct shared-memory banks (the
// cooperative kernel's layout; the one-warp kernel skews by its own topics
// per lane, see z_lane_topics).
__host__ __device__ __forceinline__ int mi(int k) { return k + (k >> 5); }
// Topics per lane of the one-warp z-step: 8 for K <= 256, 16 for K <= 512,
// 32 for K <= 1024, else 64 (two bitmap words).
__host__ __device__ __forceinline__ int z_lane_topics(int K) {
    return K <= 256 ? 8 : K <= 512 ? 16 : K <= 1024 ? 32 : 64;
}
// Shared memory of one z-step warp, in 32-bit words: m_d, then the staging
// records of the 32 tokens in flight.  The count words: K counts, the gap
// words after the lanes' slots (K / 32 + 32 of them covers (K - 1) / TPL for
// every z_lane_topics(K), and grows with K) and a leading zero, rounded up to
// 16 bytes.
__host__ __device__ __forceinline__ int z_m_words(int K) { return (K + (K >> 5) + 32 + 1 + 3) & ~3; }
constexpr int kTokRecWords = 9;     // two uint4 per token, and the offset of its word's dense q row
// ... then the warp's six 64-bit counters (z_doc_warp_t's, 16-byte aligned) and
// the document run it is working on.
constexpr int kWarpCountWords = 32;
__host__ __device__ __forceinline__ int z_warp_words(int K) { return z_m_words(K) + 32 * kTokRecWords + kWarpCountWords; }
// The counters of a warp whose shared-memory region starts at m and was sized
// for K topics: {tokens, alias draws, sum min(K_d, K_v), zero-mass tokens,
// sum |J|, tokens with K_d < K_v}, lane j updating counter j.
__device__ __forceinline__ unsigned long long *z_warp_counters(uint32_t *m, int K) {
    return reinterpret_cast<unsigned long long *>(m + z_m_words(K) + 32 * kTokRecWords);
}

// The one-warp z-step holds m_d's counts as CT: 32-bit, or 16-bit when every
// document of the launch has fewer than 65,536 tokens (half the shared
// memory, which leaves L1 more room).  The same three sizes for CT: count
// words (the counts, their gap words and a leading zero, in 32-bit words,
// rounded up to 16 bytes), the warp's whole region, and its counters.
template <typename CT>
__host__ __device__ __forceinline__ int z_count_words(int K) {
    return sizeof(CT) == 4 ? z_m_words(K) : ((K + (K >> 5) + 32 + 2 + 1) / 2 + 3) & ~3;
}
template <typename CT>
__host__ __device__ __forceinline__ int z_warp_words_t(int K) {
    return z_count_words<CT>(K) + 32 * kTokRecWords + kWarpCountWords;
}
template <typename CT>
__device__ __forceinline__ unsigned long long *z_warp_counters_t(uint32_t *m, int K) {
    return reinterpret_cast<unsigned long long *>(m + z_count_words<CT>(K) + 32 * kTokRecWords);
}
__host__ __device__ __forceinline__ int z_warp_words_n(int K, bool narrow) {
    return narrow ? z_warp_words_t<uint16_t>(K) : z_warp_words_t<uint32_t>(K);
}

// Counters of a z-step warp.  The warp-uniform ones are held one per lane
// (lane j holds counter j), which keeps five 64-bit values out of every
// lane's registers; the intersection size is summed per lane.
// Counter order: tokens, a-branch draws, sum min(K_d,K_v), zero-mass tokens,
// (lane 4 unused: sum |J| is `inter`), tokens with K_d < K_v.
struct ZCount {
    u64 mine = 0;     // this lane's warp-uniform counter
    u64 inter = 0;    // this lane's share of sum |J|
    __device__ __forceinline__ void add(int j, u64 x) {
        if ((threadIdx.x & 31) == j) mine += x;
    }
};

// One document's run: where its tokens live and where its Markov chain is.
struct DocRun {
    const int32_t *w;        // word ids, position 0 first
    int16_t *z;              // topics, updated in place
    int len;
    uint64_t seed;
    int64_t index_base;      // RNG index of position 0
    uint32_t sweep;          // sweep counter of the pass that starts at `pos`
    int pos;                 // first position to resample
    int64_t budget;          // tokens to resample in this call (passes continue past the end)
    int max_pass_end;        // stop when the pass counter reaches sweep + this many passes
    uint64_t deadline = ~0ull;   // global timer (ns): no 32-token block starts after it, but the first
};
// The run a z-step warp is working on, kept after its six counters (8-byte
// aligned: the counter area starts 16-byte aligned).
static_assert(6 * sizeof(unsigned long long) + sizeof(DocRun) <= kWarpCountWords * sizeof(uint32_t),
              "the warp's counters and document run must fit its counter area");
__device__ __forceinline__ DocRun *z_warp_run(unsigned long long *wcnt) { return reinterpret_cast<DocRun *>(wcnt + 6); }


__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Stages what depends only on token i of run r (see z_doc_warp_t for the
// record layout) and returns its current topic.
// The alias draw of the a part (Walker): slot e of the word's column keeps its
// own topic when the uniform u is below the slot's threshold, else takes the
// slot's alias topic.  Read from the packed slots when the tables carry them.
__device__ __forceinline__ int alias_outcome(const ZArgs &a, int64_t e, uint32_t u) {
    if (a.apack) {
        const uint2 s = a.apack[e];
        return guard_index(static_cast<int>(u < s.x ? s.y & 0xFFFFu : s.y >> 16), a.K, a.stats);
    }
    return guard_index(u < a.athr[e] ? a.topic[e] : a.atopic[e], a.K, a.stats);
}

__device__ __forceinline__ int stage_token(const ZArgs &a, const DocRun &r, int i, uint4 *rec2, uint32_t *drow) {
    const int wv = r.w[i];
    const int zo = guard_index(r.z[i], a.K, a.stats);
    const uint64_t t = static_cast<uint64_t>(r.index_base + i);
    const U4 x = draw(r.seed, static_cast<uint32_t>(t), static_cast<uint32_t>(t >> 32), r.sweep, TAG_Z, 0);
    const int64_t cb = a.col_ptr[wv];
    const int nw = static_cast<int>(a.col_ptr[wv + 1] - cb);
    const u64 Av = a.A[wv];
    int ta = 0;
    if (nw > 0) {
        const uint32_t sl = __umulhi(x.z, static_cast<uint32_t>(nw));
        ta = alias_outcome(a, cb + sl, x.w);
    }
    rec2[0] = make_uint4(static_cast<uint32_t>(cb),
                         static_cast<uint32_t>(static_cast<u64>(cb) >> 32) | (static_cast<uint32_t>(ta) << 16),
                         static_cast<uint32_t>(Av), static_cast<uint32_t>(Av >> 32));
    rec2[1] = make_uint4(x.x, x.y, static_cast<uint32_t>(wv), static_cast<uint32_t>(nw) | (static_cast<uint32_t>(zo) << 16));
    const int ds = a.dense_slot ? a.dense_slot[wv] : -1;
    *drow = ds >= 0 ? static_cast<uint32_t>(ds) * static_cast<uint32_t>(a.K) : 0xFFFFFFFFu;
    return zo;
}


// Adds a warp's z-step counters to the sweep's and the running totals.
// c = {tokens, a-branch draws, sum min(K_d,K_v), zero-mass tokens,
//      sum |J|, tokens with K_d < K_v}.
__device__ inline void flush_z_stats(unsigned long long *stats, const u64 (&c)[6]) {
    const int slot[6] = {ST_TOKENS, ST_ABRANCH, ST_SUMMIN, ST_ZEROMASS, ST_SUMINT, ST_DOCSIDE};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        atomicAdd(&stats[slot[i]], c[i]);
        atomicAdd(&stats[ST_COUNT + slot[i]], c[i]);
    }
}

// Zeroes, and adds to the sweep's and the running totals, a warp's counters
// kept in its shared memory (z_warp_counters).  Every lane calls them.
__device__ __forceinline__ void zero_warp_counters(unsigned long long *cnt) {
    if ((threadIdx.x & 31) < 6) cnt[threadIdx.x & 31] = 0;
    __syncwarp();
}

__device__ inline void flush_warp_counters(unsigned long long *stats, unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    // lane j's counter goes to slot {tokens, a-branch, sum min, zero mass, sum |J|, doc side}[j]
    const int slot = lane == 0 ? ST_TOKENS : lane == 1 ? ST_ABRANCH : lane == 2 ? ST_SUMMIN
                   : lane == 3 ? ST_ZEROMASS : lane == 4 ? ST_SUMINT : ST_DOCSIDE;
    __syncwarp();
    if (lane < 6) {
        const unsigned long long v = cnt[lane];
        if (v) {
            atomicAdd(&stats[slot], v);
            atomicAdd(&stats[ST_COUNT + slot], v);
        }
        cnt[lane] = 0;
    }
    __syncwarp();
}

// The same from a warp of the cooperative kernel holding its counters in a
// ZCount: lanes 0-3 and 5 hold theirs, sum |J| is summed over the lanes.
// Every lane calls it.
__device__ inline void flush_warp_z_stats(unsigned long long *stats, ZCount &c) {
    const u64 inter = warp_sum64(c.inter);
    const int lane = threadIdx.x & 31;
    const int slot[6] = {ST_TOKENS, ST_ABRANCH, ST_SUMMIN, ST_ZEROMASS, ST_SUMINT, ST_DOCSIDE};
    if (lane < 6) {
        const u64 v = lane == 4 ? inter : c.mine;
        if (v) {
            atomicAdd(&stats[slot[lane]], v);
            atomicAdd(&stats[ST_COUNT + slot[lane]], v);
        }
    }
    c = ZCount{};
}


// Largest dynamic shared memory a CTA may opt in to (device attribute).
int smem_optin();

// Opt a kernel in to the largest dynamic shared memory it can use next to
// its static shared memory.
template <typename F>
void allow_dynamic_smem(F *kernel) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    const int room = smem_optin() - static_cast<int>(fa.sharedSizeBytes);
    if (room > 0) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
}

}  // namespace pulda
