// The log-posterior diagnostic of the paper's experiments (Section 5, the
// log-posterior trace plots): the collapsed log joint of the topic indicators
// and the words, with Theta and Phi integrated out of the Dirichlet-
// multinomial LDA model,
//
//   log p(w, z | alpha, beta)
//     = sum_d [ lgamma(A) - lgamma(A + N_d) + sum_k ( lgamma(alpha_k + m_{d,k}) - lgamma(alpha_k) ) ]
//     + sum_k [ lgamma(V beta) - lgamma(V beta + n_k) + sum_v ( lgamma(beta + n_{k,v}) - lgamma(beta) ) ],
//
// A = sum_k alpha_k, n_k = sum_v n_{k,v}; terms with a zero count vanish.
// Four kernels: a table of the small-count terms, one warp per document (m_d
// in shared memory), one warp per word (the word's n column, rebuilt from z
// by the Phi-step's count pass), and one CTA that adds the per-document and
// per-word sums in a fixed order, so the same topics always give the same
// bits.
#include <algorithm>
#include <cstdint>

#include "pulda_internal.h"

namespace pulda {
namespace {

constexpr int kDiagWarps = 8;
// Most counts are small: the terms lgamma(alpha_k + c) - lgamma(alpha_k) for
// c < kTabA and lgamma(beta + n) - lgamma(beta) for n < kTabB are tabulated
// once per evaluation, with the same expression, so each term keeps its bits.
constexpr int kTabA = 256;
constexpr int kTabB = 4096;

// ta[k * kTabA + c] = lgamma(alpha_k + c) - lgamma(alpha_k);  tb[n] = lgamma(beta + n) - lgamma(beta).
__global__ void k_lp_tables(const float *alpha, int K, double beta, double *ta, double *tb) {
    const int64_t na = static_cast<int64_t>(K) * kTabA;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < na + kTabB;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (e < na) {
            const double ak = static_cast<double>(alpha[e / kTabA]);
            ta[e] = lgamma(ak + static_cast<double>(e % kTabA)) - lgamma(ak);
        } else {
            const int n = static_cast<int>(e - na);
            tb[n] = lgamma(beta + static_cast<double>(n)) - lgamma(beta);
        }
    }
}

// Butterfly sum: every lane ends with the same, order-fixed value.
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// doc_lp[d] = lgamma(A) - lgamma(A + N_d) + sum_{k: m_{d,k} > 0} (lgamma(alpha_k + m_{d,k}) - lgamma(alpha_k)).
// Documents are assigned to warps statically.
__global__ void k_lp_docs(const int64_t *doc_off, int64_t D, const int16_t *z, int K, const float *alpha, double asum,
                          const double *ta, double *doc_lp) {
    extern __shared__ uint32_t dsm[];
    const int lane = threadIdx.x & 31;
    uint32_t *m = dsm + static_cast<size_t>(threadIdx.x >> 5) * K;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int k = lane; k < K; k += 32) m[k] = 0;
    __syncwarp();
    const double lga = lgamma(asum);
    for (int64_t d = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); d < D; d += warps) {
        const int64_t b = doc_off[d], e = doc_off[d + 1];
        for (int64_t i = b + lane; i < e; i += 32) atomicAdd(&m[z[i]], 1u);
        __syncwarp();
        double t = 0.0;
        for (int k = lane; k < K; k += 32) {
            const uint32_t c = m[k];
            if (c) {
                if (c < kTabA) {
                    t += ta[static_cast<int64_t>(k) * kTabA + c];
                } else {
                    const double ak = static_cast<double>(alpha[k]);
                    t += lgamma(ak + static_cast<double>(c)) - lgamma(ak);
                }
                m[k] = 0;
            }
        }
        t = warp_sum_f64(t);
        if (lane == 0) doc_lp[d] = t + (lga - lgamma(asum + static_cast<double>(e - b)));
        __syncwarp();
    }
}

// word_lp[v] = sum_{k: n_{k,v} > 0} (lgamma(beta + n_{k,v}) - lgamma(beta)); n_k accumulated
// (integer atomics, so in any order).  Words are assigned to warps statically.
__global__ void k_lp_words(const int64_t *word_off, const uint16_t *nst_k, const uint32_t *nst_n,
                           const int32_t *nnz_n, int V, double beta, const double *tb, double *word_lp,
                           unsigned long long *nk) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const double lgb = lgamma(beta);
    for (int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < V; v += warps) {
        const int64_t b = word_off[v];
        const int cnt = nnz_n[v];
        double t = 0.0;
        for (int j = lane; j < cnt; j += 32) {
            const uint32_t n = nst_n[b + j];
            t += n < static_cast<uint32_t>(kTabB) ? tb[n] : lgamma(beta + static_cast<double>(n)) - lgb;
            atomicAdd(&nk[nst_k[b + j]], static_cast<unsigned long long>(n));
        }
        t = warp_sum_f64(t);
        if (lane == 0) word_lp[v] = t;
    }
}

// out = {total, document sum, topic sum}: each thread adds a fixed strided
// slice in order, then a fixed tree.
constexpr int kFinalThreads = 1024;
__global__ void __launch_bounds__(kFinalThreads) k_lp_final(const double *doc_lp, int64_t D, const double *word_lp,
                                                            int V, const unsigned long long *nk, int K, double beta,
                                                            double *out) {
    __shared__ double sd[kFinalThreads], st[kFinalThreads];
    const int t = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int64_t d = t; d < D; d += kFinalThreads) a += doc_lp[d];
    for (int v = t; v < V; v += kFinalThreads) b += word_lp[v];
    const double vb = static_cast<double>(V) * beta;
    const double lvb = lgamma(vb);
    for (int k = t; k < K; k += kFinalThreads) b += lvb - lgamma(vb + static_cast<double>(nk[k]));
    sd[t] = a;
    st[t] = b;
    __syncthreads();
    for (int s = kFinalThreads / 2; s > 0; s >>= 1) {
        if (t < s) {
            sd[t] += sd[t + s];
            st[t] += st[t + s];
        }
        __syncthreads();
    }
    if (t == 0) {
        out[0] = sd[0] + st[0];
        out[1] = sd[0];
        out[2] = st[0];
    }
}

int device_attr(cudaDeviceAttr what) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, what, dev);
    return v;
}

}  // namespace

size_t log_posterior_scratch_bytes(int64_t D, int V, int K) {
    return sizeof(double) * (static_cast<size_t>(D) + static_cast<size_t>(V) + 3 + static_cast<size_t>(K) * kTabA + kTabB) +
           sizeof(unsigned long long) * static_cast<size_t>(K);
}

void launch_log_posterior(const int64_t *doc_off, int64_t D, const int16_t *z, int K, const float *alpha, double asum,
                          const PhiArgs &counts, double beta, void *scratch, cudaStream_t st) {
    double *out = static_cast<double *>(scratch);
    double *doc_lp = out + 3;
    double *word_lp = doc_lp + D;
    double *ta = word_lp + counts.V;
    double *tb = ta + static_cast<size_t>(K) * kTabA;
    unsigned long long *nk = reinterpret_cast<unsigned long long *>(tb + kTabB);
    cudaMemsetAsync(nk, 0, sizeof(unsigned long long) * static_cast<size_t>(K), st);
    const int sms = std::max(1, device_attr(cudaDevAttrMultiProcessorCount));
    k_lp_tables<<<4 * sms, 256, 0, st>>>(alpha, K, beta, ta, tb);
    if (D > 0) {
        // m_d of one warp: K counts; the CTA shrinks for large K
        int warps = kDiagWarps;
        const int optin = std::max(48 * 1024, device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin));
        while (warps > 1 && static_cast<size_t>(warps) * K * sizeof(uint32_t) > static_cast<size_t>(optin)) warps >>= 1;
        const size_t smem = static_cast<size_t>(warps) * K * sizeof(uint32_t);
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_lp_docs, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lp_docs, 32 * warps, smem);
        const int64_t need = (D + warps - 1) / warps;
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(need, static_cast<int64_t>(sms) * std::max(1, per_sm))));
        k_lp_docs<<<grid, 32 * warps, smem, st>>>(doc_off, D, z, K, alpha, asum, ta, doc_lp);
    }
    const int wgrid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((counts.V + kDiagWarps - 1) / kDiagWarps, 8LL * sms)));
    k_lp_words<<<wgrid, 32 * kDiagWarps, 0, st>>>(counts.word_off, counts.nst_k, counts.nst_n, counts.nnz_n, counts.V, beta,
                                                   tb, word_lp, nk);
    k_lp_final<<<1, kFinalThreads, 0, st>>>(doc_lp, D, word_lp, counts.V, nk, K, beta, out);
}

}  // namespace pulda
