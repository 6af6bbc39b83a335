// Dirichlet Phi-step of the partially collapsed sampler (Algorithm 1), the
// method the Polya urn approximates: phi_k ~ Dir(n_k + beta) through the
// Gamma representation gamma_{k,v} ~ G(beta + n_{k,v}, 1), phi_{k,v} =
// gamma_{k,v} / sum_v gamma_{k,v} ("Efficient sampling of Phi": Gammas by
// Marsaglia and Tsang, 2000).  Every entry of the K x V matrix is drawn --
// the dense work the Polya urn's skip-ahead avoids.
//
// Readings, shared with the CPU oracle and implemented here independently:
//   Gamma draws in float, each operation rounded to float (explicit _rn
//   intrinsics); normals from the rounded-normal table; uniforms with 23
//   bits, u = (2 floor(x / 2^9) + 1) 2^-24; Philox counter (v, k, sweep,
//   TAG_GAMMA << 28 | attempt) per attempt and (v, k, sweep, TAG_GAMMA_BOOST
//   << 28) for the boost u^(1/a) of shapes a < 1; log and exp are this
//   file's own.  S_k is summed in double over chunks of kDirChunk words in
//   ascending order (each chunk in ascending v).  phi = gamma (1 / S_k) in
//   double; an entry stays in its column iff its 24-bit fixed-point weight
//   relative to the column maximum rounds to at least 1.
#include <algorithm>
#include <cstdint>

#include "device_rng.cuh"
#include "pulda_internal.h"

namespace pulda {
namespace {

constexpr int kDirBlock = 256;

// ln x for finite x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)], ln m =
// 2 atanh(s) with s = (m - 1) / (m + 1) (|s| <= 0.1716) by its series to s^9,
// ln 2 split in a short high part and a correction.
__device__ float own_logf(float x) {
    int e = 0;
    uint32_t b = __float_as_uint(x);
    if (b < 0x00800000u) {               // subnormal: scale by 2^24
        x = __fmul_rn(x, 16777216.0f);
        b = __float_as_uint(x);
        e = -24;
    }
    e += static_cast<int>(b >> 23) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > 1.41421354f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float t = __fmul_rn(s2, 0.222222224f);          // 2/9
    t = __fmul_rn(s2, __fadd_rn(0.285714298f, t));  // 2/7
    t = __fmul_rn(s2, __fadd_rn(0.400000006f, t));  // 2/5
    t = __fmul_rn(s2, __fadd_rn(0.666666687f, t));  // 2/3
    const float poly = __fmul_rn(s, __fadd_rn(2.0f, t));
    const float ef = static_cast<float>(e);
    return __fadd_rn(__fmul_rn(ef, 0.693359375f), __fadd_rn(__fmul_rn(ef, -2.12194442e-4f), poly));
}

// e^x for x <= 88: x = k ln 2 + r with |r| <= ln 2 / 2, e^r by its Taylor
// series to r^7, times 2^k (in two steps below 2^-126); 0 below -104.
__device__ float own_expf(float x) {
    if (x < -104.0f) return 0.0f;
    const float kf = floorf(__fadd_rn(__fmul_rn(x, 1.44269502f), 0.5f));
    const int k = static_cast<int>(kf);
    const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(kf, 0.693359375f)), __fmul_rn(kf, -2.12194442e-4f));
    float p = __fmul_rn(r, 0.000198412701f);       // 1/5040
    p = __fmul_rn(r, __fadd_rn(0.00138888892f, p)); // 1/720
    p = __fmul_rn(r, __fadd_rn(0.00833333377f, p)); // 1/120
    p = __fmul_rn(r, __fadd_rn(0.0416666679f, p));  // 1/24
    p = __fmul_rn(r, __fadd_rn(0.166666672f, p));   // 1/6
    p = __fmul_rn(r, __fadd_rn(0.5f, p));
    p = __fmul_rn(r, __fadd_rn(1.0f, p));
    p = __fadd_rn(1.0f, p);
    if (k >= -126) return __fmul_rn(p, __uint_as_float(static_cast<uint32_t>(k + 127) << 23));
    return __fmul_rn(__fmul_rn(p, __uint_as_float(static_cast<uint32_t>(k + 64 + 127) << 23)),
                     __uint_as_float(static_cast<uint32_t>(127 - 64) << 23));
}

__device__ __forceinline__ float unif23(uint32_t x) {
    return __fmul_rn(static_cast<float>(2u * (x >> 9) + 1u), 5.96046448e-08f);   // 2^-24
}

// gamma ~ G(a, 1), a > 0, Marsaglia and Tsang; for a < 1 the draw of
// G(a + 1) is scaled by u^(1/a).  *fail is set if no attempt was accepted.
__device__ float gamma_draw(const DevTables &T, float a, uint64_t seed, uint32_t v, uint32_t k, uint32_t sweep,
                            bool *fail) {
    const float sh = a < 1.0f ? __fadd_rn(a, 1.0f) : a;
    const float d = __fsub_rn(sh, 0.333333343f);
    const float cc = __fdiv_rn(1.0f, __fsqrt_rn(__fmul_rn(9.0f, d)));
    for (uint32_t t = 0; t < kMaxGammaTry; ++t) {
        const U4 x = draw(seed, v, k, sweep, TAG_GAMMA, t);
        const float g = __double2float_rn(gauss_draw(T, x.x, x.y));
        const float y = __fadd_rn(1.0f, __fmul_rn(cc, g));
        if (y <= 0.0f) continue;
        const float v3 = __fmul_rn(__fmul_rn(y, y), y);
        const float u = unif23(x.z);
        const float g2 = __fmul_rn(g, g);
        bool ok = u < __fsub_rn(1.0f, __fmul_rn(0.0331f, __fmul_rn(g2, g2)));
        if (!ok)
            ok = own_logf(u) < __fadd_rn(__fmul_rn(0.5f, g2),
                                         __fmul_rn(d, __fadd_rn(__fsub_rn(1.0f, v3), own_logf(v3))));
        if (ok) {
            float r = __fmul_rn(d, v3);
            if (a < 1.0f) {
                const U4 xb = draw(seed, v, k, sweep, TAG_GAMMA_BOOST, 0);
                r = __fmul_rn(r, own_expf(__fdiv_rn(own_logf(unif23(xb.x)), a)));
            }
            return r;
        }
    }
    *fail = true;
    return 0.0f;
}

// One warp per word (grid-stride): the word's n column into a dense array in
// the warp's shared memory, then gamma_{k,v} for every topic, word-major.
// Warps do not wait on one another between words.
__global__ void k_dir_gamma(PhiArgs a) {
    extern __shared__ uint32_t nsm[];
    const int K = a.K;
    const int lane = threadIdx.x & 31;
    uint32_t *nrow = nsm + static_cast<size_t>(threadIdx.x >> 5) * K;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    const uint32_t sweep = a.sweep_ptr ? *a.sweep_ptr : a.sweep;
    const float bf = static_cast<float>(a.tab.beta);
    bool fail = false;
    for (int v = blockIdx.x * wpb + (threadIdx.x >> 5); v < a.V; v += nwarps) {
        for (int k = lane; k < K; k += 32) nrow[k] = 0;
        __syncwarp();
        const int64_t b = a.word_off[v];
        for (int j = lane; j < a.nnz_n[v]; j += 32) nrow[a.nst_k[b + j]] = a.nst_n[b + j];
        __syncwarp();
        float *out = a.gam + static_cast<int64_t>(v) * K;
        for (int k = lane; k < K; k += 32) {
            const float shape = __fadd_rn(bf, static_cast<float>(nrow[k]));
            out[k] = gamma_draw(a.tab, shape, a.seed, static_cast<uint32_t>(v), static_cast<uint32_t>(k), sweep, &fail);
        }
        __syncwarp();
    }
    if (fail) atomicOr(&a.stats[ST_ERROR], ERR_GAMMA);
}

// dpart[c * K + k] = sum over the words of chunk c, in ascending order, of gamma_{k,v}.
__global__ void __launch_bounds__(kDirBlock) k_dir_rowsum_part(PhiArgs a) {
    const int K = a.K;
    const int c = blockIdx.x;
    const int v0 = c * kDirChunk, v1 = min(a.V, v0 + kDirChunk);
    for (int k = threadIdx.x; k < K; k += kDirBlock) {
        double part = 0.0;
        for (int v = v0; v < v1; ++v) part = __dadd_rn(part, static_cast<double>(a.gam[static_cast<int64_t>(v) * K + k]));
        a.dpart[static_cast<int64_t>(c) * K + k] = part;
    }
}

// S_k = the chunk sums in ascending chunk order; 1 / S_k (0 for a row of zeros).
__global__ void k_dir_rowsum_final(PhiArgs a, int n_chunks) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.K; k += gridDim.x * blockDim.x) {
        double tot = 0.0;
        for (int c = 0; c < n_chunks; ++c) tot = __dadd_rn(tot, a.dpart[static_cast<int64_t>(c) * a.K + k]);
        a.Sd[k] = tot;
        a.invS[k] = tot > 0.0 ? __ddiv_rn(1.0, tot) : 0.0;
        a.invSf[k] = __double2float_rn(a.invS[k]);
    }
}

// One warp per word: phi = gamma (1/S_k) in double; the column maximum fixes
// the fixed-point scale 2^(24 - e); entries whose weight rounds to 0 are
// dropped, the rest staged in ascending topic order (cst_k, cst_c = the
// draw's bits).  FP64 is scarce on this GPU, so a float product screens every
// entry (relative error below 2^-22): the maximum is taken exactly over the
// entries within 2^-12 of the float maximum, and an entry is decided by the
// double test only within 0.1% of the threshold 2^(e-25).  Tiny columns (float
// maximum or threshold below 2^-100, where float products lose precision) take
// the double path throughout.  The decisions are those of the double test.
__global__ void k_dir_select(PhiArgs a) {
    const int lane = threadIdx.x & 31;
    const int K = a.K;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const float kTiny = 7.88860905e-31f;      // 2^-100
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < a.V; v += nwarps) {
        const float *g = a.gam + static_cast<int64_t>(v) * K;
        float fmax = 0.0f;
        for (int k = lane; k < K; k += 32) fmax = fmaxf(fmax, __fmul_rn(g[k], a.invSf[k]));
#pragma unroll
        for (int o = 16; o; o >>= 1) fmax = fmaxf(fmax, __shfl_xor_sync(0xFFFFFFFFu, fmax, o));
        const bool exact_all = fmax < kTiny;
        const float fcut = __fmul_rn(fmax, 0.999755859f);       // 1 - 2^-12
        double pmax = 0.0;
        for (int k = lane; k < K; k += 32) {
            if (exact_all || __fmul_rn(g[k], a.invSf[k]) >= fcut) {
                const double p = __dmul_rn(static_cast<double>(g[k]), a.invS[k]);
                pmax = p > pmax ? p : pmax;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const double y = __shfl_xor_sync(0xFFFFFFFFu, pmax, o);
            pmax = y > pmax ? y : pmax;
        }
        int kept = 0;
        if (pmax > 0.0) {
            const long long bits = __double_as_longlong(pmax);
            const int e = static_cast<int>((bits >> 52) & 0x7FF) - 1022;
            const double scale = __longlong_as_double(static_cast<long long>(1023 + 24 - e) << 52);
            // threshold 2^(e-25) in float, when it is a normal float well above the subnormals
            const bool screen = !exact_all && e - 25 >= -100;
            const float thr = screen ? __uint_as_float(static_cast<uint32_t>(e - 25 + 127) << 23) : 0.0f;
            const float hi = __fmul_rn(thr, 1.001f), lo = __fmul_rn(thr, 0.999f);
            const int64_t dst = static_cast<int64_t>(v) * K;
            for (int k0 = 0; k0 < K; k0 += 32) {
                const int k = k0 + lane;
                bool keep = false;
                float gk = 0.0f;
                if (k < K) {
                    gk = g[k];
                    const float pf = screen ? __fmul_rn(gk, a.invSf[k]) : 0.0f;
                    if (screen && pf >= hi) {
                        keep = true;
                    } else if (!screen || pf > lo) {
                        const double p = __dmul_rn(static_cast<double>(gk), a.invS[k]);
                        keep = floor(__dadd_rn(__dmul_rn(p, scale), 0.5)) >= 1.0;
                    }
                }
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
                if (keep) {
                    const int at = kept + __popc(bal & ((1u << lane) - 1u));
                    a.cst_k[dst + at] = static_cast<uint16_t>(k);
                    a.cst_c[dst + at] = __float_as_uint(gk);
                }
                kept += __popc(bal);
            }
        }
        if (lane == 0) a.nnz_c[v] = kept;
    }
}

int sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

size_t dir_part_count(int V, int K) {
    return static_cast<size_t>((V + kDirChunk - 1) / kDirChunk) * static_cast<size_t>(K);
}

void launch_dir_phi(const PhiArgs &a, cudaStream_t st) {
    const int n = sms();
    // one warp per word, its n row (K counts) in shared memory: up to 8 warps
    // per CTA within 96 KB (one warp of up to 64 KB for the largest K)
    int wpb = 8;
    while (wpb > 1 && static_cast<size_t>(wpb) * a.K * sizeof(uint32_t) > 96 * 1024) wpb >>= 1;
    const size_t smem = static_cast<size_t>(wpb) * a.K * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncSetAttribute(k_dir_gamma, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    }
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((a.V + wpb - 1) / wpb, 16LL * n)));
    k_dir_gamma<<<grid, 32 * wpb, smem, st>>>(a);
    const int n_chunks = (a.V + kDirChunk - 1) / kDirChunk;
    k_dir_rowsum_part<<<n_chunks, kDirBlock, 0, st>>>(a);
    k_dir_rowsum_final<<<(a.K + 255) / 256, 256, 0, st>>>(a, n_chunks);
    k_dir_select<<<std::max(1, std::min((a.V + 7) / 8, 8 * n)), 256, 0, st>>>(a);
}

}  // namespace pulda
