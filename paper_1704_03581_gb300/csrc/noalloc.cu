// pulda_infer_noalloc: fold-in of new documents that allocates no memory.
//
// Some callers cannot call cudaMalloc (or anything that does): a serving
// process whose device memory is carved up once at start-up and must not
// grow, a memory-capped tenant on a shared GPU, or a host thread that must not
// block on the allocator's device-wide synchronisation in the middle of a
// latency-critical loop.  pulda_infer allocates temporaries for every call;
// this entry point takes the caller's device buffers for inputs and outputs and
// keeps the little scratch the z-step kernel needs (its work counter, its
// counters and the document schedule) in one file-scope device array instead.
//
// That array is static device memory of the library: every GPU that loads
// the library holds it until the process exits, and every call on a device
// shares it.  So calls that overlap on the GPU (from two host threads or two
// streams) race on it and must be serialised by the caller.  What must start
// at zero is cleared by each call.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/pulda.h"
#include "pulda_internal.h"

namespace pulda {
namespace {

// Largest number of documents one call may carry.
constexpr int64_t kNoAllocMaxDocs = 65536;

// Layout of the scratch array (bytes, each part 256-byte aligned).
constexpr size_t kOffStats = 0;                                       // u64[ST_TOTAL_SLOTS]
constexpr size_t kOffWork = 256;                                      // int[4]: z-step work counter
constexpr size_t kOffFlag = 512;                                      // u64[2]: first bad token, first bad document
constexpr size_t kOffOrder = 768;                                     // int32[kNoAllocMaxDocs]
constexpr size_t kScratchBytes = kOffOrder + sizeof(int32_t) * kNoAllocMaxDocs;   // 262,912 bytes
static_assert(ST_TOTAL_SLOTS * sizeof(unsigned long long) <= kOffWork, "the counters overlap the work counter");
static_assert(4 * sizeof(int) <= kOffFlag - kOffWork, "the work counters overlap the input check");
static_assert(2 * sizeof(unsigned long long) <= kOffOrder - kOffFlag, "the input check overlaps the schedule");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch on each device, found once per device.
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// One-time set-up per device, with that device current (the caller checks
// that it is the handle's): look up where the array lives on it.  The
// host-side symbol g_noalloc_scratch is only a stand-in and must never be
// handed to a kernel.
cudaError_t scratch_on_device(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    cudaError_t e = cudaSuccess;
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Checks the caller's device inputs (ids in [0, V), offsets nondecreasing from
// 0 to N) and writes the identity document schedule.  first[0] becomes the
// smallest position of a word id outside [0, V), first[1] the smallest
// document with bad offsets; both start at ~0 (none).
__global__ void k_noalloc_check(const int32_t *w, int64_t N, const int64_t *off, int64_t D, int V,
                                unsigned long long *first, int32_t *order) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    for (int64_t i = t0; i < N; i += stride)
        if (w[i] < 0 || w[i] >= V) atomicMin(&first[0], static_cast<unsigned long long>(i));
    for (int64_t d = t0; d < D; d += stride) {
        order[d] = static_cast<int32_t>(d);
        const int64_t a = off[d], b = off[d + 1];
        if (a < 0 || b < a || b > N || (d == 0 && a != 0) || (d == D - 1 && b != N) || b - a > (int64_t(1) << 22))
            atomicMin(&first[1], static_cast<unsigned long long>(d));
    }
}

}  // namespace
}  // namespace pulda

using namespace pulda;

extern "C" pulda_status pulda_infer_noalloc(pulda_handle *h, const int32_t *word_ids_dev,
                                            const int64_t *doc_offsets_dev, int64_t D_new, int64_t N_new,
                                            int32_t n_sweeps, uint64_t seed, int16_t *z_out_dev) {
    HandleView hv{};
    if (!handle_view(h, &hv)) return PULDA_ERR_INVALID;
    if (!hv.have_phi)
        return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_INVALID, "no Phi drawn yet: run a sweep first"));
    if (D_new < 0 || D_new > kNoAllocMaxDocs)
        return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_INVALID,
            "pulda_infer_noalloc takes at most 65536 documents per call (its scratch is fixed)"));
    if (N_new < 0 || N_new >= (int64_t(1) << 31))
        return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_INVALID, "N_new must be in [0, 2^31)"));
    if (n_sweeps < 0) return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_INVALID, "n_sweeps must be >= 0"));
    if (D_new == 0) return PULDA_OK;
    if (!word_ids_dev || !doc_offsets_dev || !z_out_dev)
        return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_INVALID, "a device pointer is NULL"));
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_CUDA, cudaGetErrorString(e)));
    if (dev != hv.device) {
        char msg[160];
        snprintf(msg, sizeof msg, "the calling thread's current device (%d) is not the handle's (%d)", dev, hv.device);
        return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_INVALID, msg));
    }
    unsigned char *scratch = nullptr;
    e = scratch_on_device(dev, &scratch);
    if (e != cudaSuccess)
        return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_CUDA, cudaGetErrorString(e)));
    cudaStream_t st = hv.stream;
    auto *stats = reinterpret_cast<unsigned long long *>(scratch + kOffStats);
    auto *work = reinterpret_cast<int *>(scratch + kOffWork);
    auto *first = reinterpret_cast<unsigned long long *>(scratch + kOffFlag);
    auto *order = reinterpret_cast<int32_t *>(scratch + kOffOrder);
    // the array keeps the previous call's contents: clear what counts from
    // zero, and set the input check's "first bad index" slots to ~0 (none)
    e = cudaMemsetAsync(scratch, 0, kOffFlag, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(first, 0xFF, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        k_noalloc_check<<<64, 256, 0, st>>>(word_ids_dev, N_new, doc_offsets_dev, D_new, hv.V, first, order);
        e = cudaGetLastError();
    }
    unsigned long long hfirst[2] = {~0ull, ~0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hfirst, first, sizeof hfirst, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_CUDA, cudaGetErrorString(e)));
    if (hfirst[1] != ~0ull) {
        char msg[200];
        snprintf(msg, sizeof msg, "doc offsets must rise from 0 to N_new, each document at most 2^22 tokens "
                 "(first bad document: %llu)", hfirst[1]);
        return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_INVALID, msg));
    }
    if (hfirst[0] != ~0ull) {
        char msg[160];
        snprintf(msg, sizeof msg, "the word id at token %llu is outside [0, %d)", hfirst[0], hv.V);
        return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_INVALID, msg));
    }
    launch_init_z(N_new, hv.K, seed, 0, z_out_dev, st);
    ZArgs a = hv.zargs;
    a.doc_off = doc_offsets_dev;
    a.doc_order = order;
    a.D = D_new;
    a.w = word_ids_dev;
    a.z = z_out_dev;
    a.seed = seed;
    a.index_base = 0;
    a.work = work;
    a.stats = stats;
    for (int32_t sw = 1; sw <= n_sweeps && e == cudaSuccess; ++sw) {
        e = cudaMemsetAsync(work, 0, sizeof(int), st);
        a.sweep = static_cast<uint32_t>(sw);
        if (e == cudaSuccess) {
            launch_z_step(a, hv.z_warps, hv.z_grid, st);
            e = cudaGetLastError();
        }
    }
    unsigned long long err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, stats + ST_ERROR, sizeof err, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_CUDA, cudaGetErrorString(e)));
    if (err) return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_CUDA, "z-step invariant violated"));
    return PULDA_OK;
}
