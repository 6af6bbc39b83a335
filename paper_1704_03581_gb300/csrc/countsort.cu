// The count rebuild n_{k,v} = #{i : z_i = k, w_i = v} (notation table) by
// sorting, beside the per-word shared-memory histograms of kernels.cu: every
// token's key w_i K + z_i is sorted (least-significant-digit radix sort,
// 8-bit digits, stable), each run of equal keys is one nonzero n_{k,v} with
// the run's length, and the runs of word v, already in ascending topic order,
// are its n column at word_off[v].  The Phi-step's draw pass then reads the
// columns instead of histogramming.  Exact integers either way: the columns
// are bit-identical to the histograms'.
#include <algorithm>
#include <cstdint>

#include "pulda_internal.h"
#include "checks.cuh"

namespace pulda {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;                               // keys per thread
constexpr int kSortTile = kSortThreads * kSortRounds;         // keys per CTA
constexpr int kWarpKeys = 32 * kSortRounds;                   // a warp's run of consecutive keys
constexpr int kBins = 256;
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_sort_keys(const int32_t *w, const int16_t *z, int64_t N, int K, uint32_t *key,
                            unsigned long long *stats) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < N; i += stride)
        key[i] = static_cast<uint32_t>(w[i]) * static_cast<uint32_t>(K) +
                 static_cast<uint32_t>(guard_index(z[i], K, stats));
}

// counts[d * nb + b] = keys of tile b whose digit at `shift` is d.
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *key, int64_t N, int shift,
                                                             uint32_t *counts) {
    __shared__ uint32_t h[kBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
#pragma unroll 4
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + static_cast<int64_t>(r) * kSortThreads + threadIdx.x;
        if (i < N) atomicAdd(&h[(key[i] >> shift) & (kBins - 1)], 1u);
    }
    __syncthreads();
    counts[static_cast<int64_t>(threadIdx.x) * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of tile b: key j of the tile (in index order) goes to
// offsets[d * nb + b] + its rank among the tile's keys of digit d.  Warp w
// ranks its run of kWarpKeys consecutive keys 32 at a time (peers by
// __match_any_sync); the warps' runs are then placed in warp order.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t *in, uint32_t *out, int64_t N,
                                                                int shift, const uint32_t *offsets) {
    __shared__ uint32_t wcnt[kSortWarps][kBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kBins; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile + static_cast<int64_t>(warp) * kWarpKeys;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t k[kSortRounds];
    uint32_t rank[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + static_cast<int64_t>(r) * 32 + lane;
        const bool valid = i < N;
        k[r] = valid ? in[i] : 0u;
        const uint32_t d = (k[r] >> shift) & (kBins - 1);
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, valid ? d : kBins + lane);
        const uint32_t before = wcnt[warp][d];            // read by every peer before the leader adds
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    {   // each digit's run of warps: exclusive offsets within the tile
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + static_cast<int64_t>(r) * 32 + lane;
        if (i < N) {
            const uint32_t d = (k[r] >> shift) & (kBins - 1);
            out[offsets[static_cast<int64_t>(d) * gridDim.x + blockIdx.x] + wcnt[warp][d] + rank[r]] = k[r];
        }
    }
}

// ---------------------------------------------------------------- exclusive scan (uint32, in place)
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *tmp, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < kScanThreads / 32 ? tmp[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < kScanThreads / 32) tmp[lane] = ti - t;
        if (lane == 31) tmp[kScanThreads / 32] = ti;
    }
    __syncthreads();
    const uint32_t r = tmp[warp] + incl - v;
    total = tmp[kScanThreads / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *data, int64_t n, uint32_t *sums) {
    __shared__ uint32_t tmp[kScanThreads / 32 + 1];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < n) s += data[base + j];
    uint32_t total;
    block_excl_scan_u32(s, tmp, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One CTA: the block sums' exclusive scan, in place, 4096 at a time with a carry.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t *sums, int64_t nb) {
    __shared__ uint32_t tmp[kScanThreads / 32 + 1];
    uint32_t carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += kScanTile) {
        const int64_t base = c0 + static_cast<int64_t>(threadIdx.x) * kScanItems;
        uint32_t v[kScanItems];
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            v[j] = base + j < nb ? sums[base + j] : 0u;
            s += v[j];
        }
        uint32_t total;
        uint32_t run = carry + block_excl_scan_u32(s, tmp, total);
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            if (base + j < nb) sums[base + j] = run;
            run += v[j];
        }
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(uint32_t *data, int64_t n, const uint32_t *sums) {
    __shared__ uint32_t tmp[kScanThreads / 32 + 1];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < n ? data[base + j] : 0u;
        s += v[j];
    }
    uint32_t total;
    uint32_t run = sums[blockIdx.x] + block_excl_scan_u32(s, tmp, total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) data[base + j] = run;
        run += v[j];
    }
}

void excl_scan_u32(uint32_t *data, int64_t n, uint32_t *sums, cudaStream_t st) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb <= 0) return;
    k_scan_reduce<<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(data, n, sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, nb);
    k_scan_apply<<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(data, n, sums);
}

// ---------------------------------------------------------------- runs -> n columns
// flag[i] = 1 where a run of equal keys starts (flag[N] = 0).
__global__ void k_run_flags(const uint32_t *key, int64_t N, uint32_t *flag) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i <= N; i += stride)
        flag[i] = i < N && (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
}

// After the scan rid[i] = runs starting before i: each run's first position.
__global__ void k_run_starts(const uint32_t *key, const uint32_t *rid, int64_t N, uint32_t *start) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < N; i += stride)
        if (i == 0 || key[i] != key[i - 1]) start[rid[i]] = static_cast<uint32_t>(i);
}

// Run r of word v (the sorted keys of word v occupy [word_off[v], word_off[v+1]))
// is entry r - rid[word_off[v]] of its n column: (topic, run length).
__global__ void k_run_emit(const uint32_t *key, const uint32_t *rid, const uint32_t *start, int64_t N, int K,
                           const int64_t *word_off, uint16_t *nst_k, uint32_t *nst_n) {
    const int64_t R = rid[N];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < R; r += stride) {
        const uint32_t i = start[r];
        const uint32_t e = r + 1 < R ? start[r + 1] : static_cast<uint32_t>(N);
        const uint32_t kk = key[i];
        const int v = static_cast<int>(kk / static_cast<uint32_t>(K));
        const int64_t wb = word_off[v];
        const int64_t j = r - rid[wb];
        nst_k[wb + j] = static_cast<uint16_t>(kk - static_cast<uint32_t>(v) * static_cast<uint32_t>(K));
        nst_n[wb + j] = e - i;
    }
}

__global__ void k_run_nnz(const uint32_t *rid, const int64_t *word_off, int V, int32_t *nnz_n) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride)
        nnz_n[v] = static_cast<int32_t>(rid[word_off[v + 1]] - rid[word_off[v]]);
}

int grid_for(int64_t n, int threads) {
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152LL * 16)));
}

}  // namespace

size_t count_sort_scratch_words(int64_t N) {
    const int64_t nb = (N + kSortTile - 1) / kSortTile;
    const int64_t scan_n = std::max<int64_t>(N + 1, kBins * nb);
    return static_cast<size_t>(3 * N + 2 + kBins * nb + (scan_n + kScanTile - 1) / kScanTile + 1);
}

void launch_count_sort(const int32_t *w, const int16_t *z, int64_t N, int K, int V, const int64_t *word_off,
                       uint16_t *nst_k, uint32_t *nst_n, int32_t *nnz_n, uint32_t *scratch,
                       unsigned long long *stats, cudaStream_t st) {
    if (N <= 0) {
        cudaMemsetAsync(nnz_n, 0, sizeof(int32_t) * V, st);
        return;
    }
    const int64_t nb = (N + kSortTile - 1) / kSortTile;
    uint32_t *a = scratch;                    // keys
    uint32_t *b = a + N;                      // keys (other buffer)
    uint32_t *c = b + N;                      // flags -> run ids [N + 1], then run starts
    uint32_t *counts = c + N + 1;             // [kBins * nb]
    uint32_t *sums = counts + kBins * nb;     // scan block sums
    k_sort_keys<<<grid_for(N, 256), 256, 0, st>>>(w, z, N, K, a, stats);
    const uint64_t top = static_cast<uint64_t>(V) * static_cast<uint64_t>(K);
    int bits = 1;
    while (bits < 32 && (uint64_t(1) << bits) < top) ++bits;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<static_cast<unsigned>(nb), kSortThreads, 0, st>>>(a, N, shift, counts);
        excl_scan_u32(counts, kBins * nb, sums, st);
        k_radix_scatter<<<static_cast<unsigned>(nb), kSortThreads, 0, st>>>(a, b, N, shift, counts);
        std::swap(a, b);
    }
    k_run_flags<<<grid_for(N + 1, 256), 256, 0, st>>>(a, N, c);
    excl_scan_u32(c, N + 1, sums, st);
    // run starts go to b (no longer needed as keys)
    k_run_starts<<<grid_for(N, 256), 256, 0, st>>>(a, c, N, b);
    k_run_emit<<<grid_for(N, 256), 256, 0, st>>>(a, c, b, N, K, word_off, nst_k, nst_n);
    k_run_nnz<<<grid_for(V, 256), 256, 0, st>>>(c, word_off, V, nnz_n);
}

}  // namespace pulda
