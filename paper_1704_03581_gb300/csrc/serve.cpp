// Continuous-batching fold-in server: new documents, of uneven length,
// resampled against a fixed Phi (Algorithm 2's z-step with Phi held) as they
// arrive.  A worker thread owns the GPU side: it admits waiting requests while
// a slot and a contiguous range of the token arena are free (memory-based
// admission, first come first served), advances every admitted request by up
// to `slice` tokens per launch -- one warp per request (one CTA of the
// cooperative z-step per long request, on a second stream), passes continuing
// within the launch -- and hands finished requests back.  With the automatic
// slice a launch instead runs every request for a 2 ms window, so each
// advances as far as its own speed allows.  Each request's
// random streams are keyed by its own seed and token positions, so its result
// does not depend on which other requests shared the GPU with it: it equals
// pulda_infer on that document alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include <time.h>

#include "../../include/pulda.h"
#include "handle.h"
#include "pulda_internal.h"

using namespace pulda;

namespace {

int64_t now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return static_cast<int64_t>(ts.tv_sec) * 1000000000LL + ts.tv_nsec;
}

struct Request {
    uint64_t id = 0, seed = 0;
    std::vector<int32_t> words;
    int32_t n_sweeps = 0;
    int16_t *z_out = nullptr;
    int64_t submit_ns = 0;
    int64_t off = -1;
};

// First-fit allocator of contiguous token ranges of the arena.
class Arena {
public:
    explicit Arena(int64_t n) { if (n > 0) free_[0] = n; }
    int64_t alloc(int64_t len) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                const int64_t off = it->first, rest = it->second - len;
                free_.erase(it);
                if (rest > 0) free_[off + len] = rest;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, int64_t len) {
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }
private:
    std::map<int64_t, int64_t> free_;
};

constexpr size_t kMaxPending = size_t(1) << 22;
#ifndef PULDA_SERVE_COOP_GATE
#define PULDA_SERVE_COOP_GATE 8
#endif
constexpr int64_t kServeCoopGate = PULDA_SERVE_COOP_GATE;   // cooperative while n_active * this <= resident warps

}  // namespace

struct pulda_server {
    pulda_handle *h = nullptr;
    int device = 0;
    cudaStream_t stream = nullptr, stream2 = nullptr;   // the cooperative launch, the one-warp launch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int64_t budget = 0, slice = 0;
    int64_t coop_len = 0;                 // requests at least this long go to the cooperative kernel (0 = none)
    uint64_t window_ns = 0;               // automatic slice: the launch's time window
    int32_t max_slots = 0;
    int z_warps = 8, grid = 1, coop_grid = 1;
    ZArgs tabs{};
    // device state
    int32_t *arena_w = nullptr;
    int16_t *arena_z = nullptr;
    ServeSlot *d_slots = nullptr;
    int32_t *d_active = nullptr;
    int *d_work = nullptr;
    unsigned long long *d_stats = nullptr;
    ServeSlot *h_slots = nullptr;        // pinned: slot states read back after each launch
    ServeSlot *h_new = nullptr;          // pinned: entries of newly admitted slots
    int32_t *h_active = nullptr;         // pinned: the active list of the next launch
    std::vector<int32_t> h_slots_len;    // tokens of each slot's request
    int32_t *pin_w = nullptr;            // pinned mirror of the arena's word ids
    int16_t *pin_z = nullptr;            // pinned mirror of the arena's topics
    bool auto_slice = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // counters: iterations, admitted, completed, token steps, kernel ns, current slice, max active
    int64_t ctr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // host state
    Arena arena{0};
    std::vector<Request> slot_req;
    std::vector<int32_t> free_slots, active;
    std::deque<Request> pending;
    std::deque<pulda_result> done;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::string err;
    pulda_status err_status = PULDA_OK;
    std::thread worker;
};

namespace {

bool check(pulda_server *s, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    std::lock_guard<std::mutex> lock(s->mu);
    s->err = std::string(what) + ": " + cudaGetErrorString(e);
    s->err_status = PULDA_ERR_CUDA;
    s->cv_done.notify_all();
    return false;
}

// Moves waiting requests into free slots while the arena has room (first come
// first served) and enqueues their uploads; called with s->mu held.
void admit_locked(pulda_server *s, std::vector<int32_t> &newly) {
    while (!s->pending.empty() && !s->free_slots.empty()) {
        Request &r = s->pending.front();
        const int64_t len = static_cast<int64_t>(r.words.size());
        const int64_t off = s->arena.alloc(len);
        if (off < 0) break;                         // wait for memory to free up
        const int32_t slot = s->free_slots.back();
        s->free_slots.pop_back();
        r.off = off;
        std::memcpy(s->pin_w + off, r.words.data(), sizeof(int32_t) * len);
        s->h_new[slot] = ServeSlot{off, static_cast<int32_t>(len), 0, 0, static_cast<uint32_t>(1 + r.n_sweeps), r.seed};
        s->h_slots_len[slot] = static_cast<int32_t>(len);
        s->slot_req[slot] = std::move(r);
        s->pending.pop_front();
        newly.push_back(slot);
    }
}

bool upload(pulda_server *s, const std::vector<int32_t> &newly) {
    for (int32_t slot : newly) {
        const ServeSlot &e = s->h_new[slot];
        if (!check(s, cudaMemcpyAsync(s->arena_w + e.off, s->pin_w + e.off, sizeof(int32_t) * e.len,
                                      cudaMemcpyHostToDevice, s->stream), "upload of a request")) return false;
        if (!check(s, cudaMemcpyAsync(s->d_slots + slot, s->h_new + slot, sizeof(ServeSlot), cudaMemcpyHostToDevice,
                                      s->stream), "upload of a slot")) return false;
    }
    return true;
}

void worker_loop(pulda_server *s) {
    cudaSetDevice(s->device);
    std::vector<int32_t> newly, finished, still;
    for (;;) {
        // requests admitted during the previous launch are already uploaded;
        // if nothing runs, wait for arrivals
        if (s->active.empty() && newly.empty()) {
            std::unique_lock<std::mutex> lock(s->mu);
            for (;;) {
                admit_locked(s, newly);
                if (!newly.empty()) break;
                if (s->stop && s->pending.empty()) return;
                s->cv_work.wait_for(lock, std::chrono::milliseconds(2));
            }
            lock.unlock();
            if (!upload(s, newly)) return;
        }
        for (int32_t slot : newly) s->active.push_back(slot);
        newly.clear();
        const int n = static_cast<int>(s->active.size());
        // long requests first (the cooperative kernel's), then the others.  A
        // cooperative token costs about four times the issue slots of a
        // one-warp token, which pays while the SMs have idle issue slots: only
        // while the active requests fill at most an eighth of the resident warps
        // (measured: at a quarter, 20k requests/s doubled p50).
        const bool coop = s->coop_len > 0 &&
                          static_cast<int64_t>(n) * kServeCoopGate <= static_cast<int64_t>(s->grid) * s->z_warps;
        int nc = 0;
        for (int32_t slot : s->active)
            if (coop && s->h_slots_len[slot] >= s->coop_len) s->h_active[nc++] = slot;
        int j = nc;
        bool narrow = true;     // every request on the one-warp kernel fits 16-bit counts
        for (int32_t slot : s->active)
            if (!(coop && s->h_slots_len[slot] >= s->coop_len)) {
                s->h_active[j++] = slot;
                narrow = narrow && s->h_slots_len[slot] <= kNarrowMaxLen;
            }
        if (!check(s, cudaMemcpyAsync(s->d_active, s->h_active, sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                                      s->stream), "upload of the active list")) return;
        cudaEventRecord(s->ev0, s->stream);
        if (nc > 0) {
            cudaEventRecord(s->ev_fork, s->stream);
            launch_serve_step_coop(s->tabs, s->d_slots, s->d_active, nc, s->arena_w, s->arena_z, s->slice,
                                   s->d_work + 1, s->coop_grid, s->window_ns, s->stream);
            cudaStreamWaitEvent(s->stream2, s->ev_fork, 0);
            launch_serve_step(s->tabs, s->d_slots, s->d_active + nc, n - nc, s->arena_w, s->arena_z, s->slice,
                              s->d_work, s->z_warps, s->grid, s->window_ns, narrow, s->stream2);
            cudaEventRecord(s->ev_join, s->stream2);
            cudaStreamWaitEvent(s->stream, s->ev_join, 0);
        } else {
            launch_serve_step(s->tabs, s->d_slots, s->d_active, n, s->arena_w, s->arena_z, s->slice, s->d_work,
                              s->z_warps, s->grid, s->window_ns, narrow, s->stream);
        }
        if (!check(s, cudaGetLastError(), "serving launch")) return;
        cudaEventRecord(s->ev1, s->stream);
        if (!check(s, cudaMemcpyAsync(s->h_slots, s->d_slots, sizeof(ServeSlot) * s->max_slots, cudaMemcpyDeviceToHost,
                                      s->stream), "slot read-back")) return;
        // admit and upload the next requests while the launch runs
        {
            std::lock_guard<std::mutex> lock(s->mu);
            admit_locked(s, newly);
        }
        if (!upload(s, newly)) return;
        if (!check(s, cudaStreamSynchronize(s->stream), "serving step")) return;
        float kms = 0.f;
        cudaEventElapsedTime(&kms, s->ev0, s->ev1);
        s->ctr[0] += 1;
        s->ctr[4] += static_cast<int64_t>(kms * 1e6);
        s->ctr[6] = std::max<int64_t>(s->ctr[6], n);
        s->ctr[5] = s->slice;
        finished.clear();
        still.clear();
        for (int32_t slot : s->active) {
            const ServeSlot &e = s->h_slots[slot];
            if (e.sweep >= e.sweep_end) {
                if (!check(s, cudaMemcpyAsync(s->pin_z + e.off, s->arena_z + e.off, sizeof(int16_t) * e.len,
                                              cudaMemcpyDeviceToHost, s->stream), "result copy")) return;
                finished.push_back(slot);
            } else {
                still.push_back(slot);
            }
        }
        s->active.swap(still);
        if (finished.empty()) continue;
        unsigned long long err = 0;
        if (!check(s, cudaMemcpyAsync(&err, s->d_stats + ST_ERROR, sizeof err, cudaMemcpyDeviceToHost, s->stream),
                   "error read-back")) return;
        if (!check(s, cudaStreamSynchronize(s->stream), "result copies")) return;
        for (int32_t slot : finished) {
            Request &r = s->slot_req[slot];
            if (r.z_out) std::memcpy(r.z_out, s->pin_z + r.off, sizeof(int16_t) * r.words.size());
        }
        const int64_t t = now_ns();
        std::lock_guard<std::mutex> lock(s->mu);
        for (int32_t slot : finished) {
            Request &r = s->slot_req[slot];
            pulda_result res{};
            res.req_id = r.id;
            res.status = err ? PULDA_ERR_CUDA : PULDA_OK;
            res.len = static_cast<int32_t>(r.words.size());
            res.submit_ns = r.submit_ns;
            res.done_ns = t;
            s->done.push_back(res);
            s->ctr[2] += 1;
            s->ctr[3] += static_cast<int64_t>(r.words.size()) * (r.n_sweeps);
            s->arena.release(r.off, static_cast<int64_t>(r.words.size()));
            r = Request();
            s->free_slots.push_back(slot);
        }
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

pulda_status pulda_serve_open(pulda_handle *h, int64_t token_budget, int32_t max_slots, int64_t slice_tokens,
                              pulda_server **out) {
    if (!h || !out) return PULDA_ERR_INVALID;
    *out = nullptr;
    if (!h->have_phi) return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_INVALID, "no Phi drawn yet: run a sweep first"));
    if (token_budget < 1 || max_slots < 1 || slice_tokens < 0)
        return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_INVALID,
                                                     "token_budget and max_slots must be >= 1, slice_tokens >= 0"));
    // the server's launches run on its own streams: the sweeps still queued on
    // the handle's stream must have written Phi and its tables first
    const pulda_status ready = pulda_sync(h);
    if (ready != PULDA_OK) return ready;
    pulda_server *s = new pulda_server();
    s->h = h;
    s->budget = token_budget;
    s->auto_slice = slice_tokens == 0;
    // automatic: launches of about 2 ms (long enough to amortise the loop,
    // short enough that new requests start soon), however far each request gets
    s->slice = slice_tokens == 0 ? (int64_t(1) << 22) : slice_tokens;
    s->window_ns = slice_tokens == 0 ? 2000000ull : 0ull;
    s->coop_len = h->opt.coop_min_len < 0 ? 0 : (h->opt.coop_min_len > 0 ? h->opt.coop_min_len : kServeCoopAuto);
    s->max_slots = max_slots;
    s->h_slots_len.assign(max_slots, 0);
    s->arena = Arena(token_budget);
    s->slot_req.resize(max_slots);
    for (int32_t i = max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    cudaGetDevice(&s->device);
    auto bad = [&](cudaError_t e, const char *what) {
        handle_fail(h, e == cudaErrorMemoryAllocation ? PULDA_ERR_OOM : PULDA_ERR_CUDA, what);
        pulda_serve_close(s);
        return e == cudaErrorMemoryAllocation ? PULDA_ERR_OOM : PULDA_ERR_CUDA;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete s; return static_cast<pulda_status>(handle_fail(h, PULDA_ERR_CUDA, "stream creation failed")); }
    if ((e = cudaStreamCreateWithFlags(&s->stream2, cudaStreamNonBlocking)) != cudaSuccess) return bad(e, "stream creation failed");
    if ((e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming)) != cudaSuccess)
        return bad(e, "event creation failed");
    // device buffers through the handle's allocator (the caller's, if it set one)
    auto dalloc = [&](auto **p, size_t bytes) {
        void *q = nullptr;
        const cudaError_t r = dev_alloc(h->opt, s->stream, bytes, &q, false);
        *p = static_cast<std::remove_pointer_t<std::remove_reference_t<decltype(p)>>>(q);
        return r;
    };
    if ((e = dalloc(&s->arena_w, sizeof(int32_t) * token_budget)) != cudaSuccess) return bad(e, "arena allocation failed");
    if ((e = dalloc(&s->arena_z, sizeof(int16_t) * token_budget)) != cudaSuccess) return bad(e, "arena allocation failed");
    if ((e = dalloc(&s->d_slots, sizeof(ServeSlot) * max_slots)) != cudaSuccess) return bad(e, "slot table allocation failed");
    if ((e = dalloc(&s->d_active, sizeof(int32_t) * max_slots)) != cudaSuccess) return bad(e, "slot table allocation failed");
    if ((e = dalloc(&s->d_work, sizeof(int) * 4)) != cudaSuccess) return bad(e, "allocation failed");
    if ((e = dalloc(&s->d_stats, sizeof(unsigned long long) * ST_TOTAL_SLOTS)) != cudaSuccess) return bad(e, "allocation failed");
    if ((e = cudaMallocHost(&s->h_slots, sizeof(ServeSlot) * max_slots)) != cudaSuccess) return bad(e, "pinned allocation failed");
    if ((e = cudaMallocHost(&s->h_new, sizeof(ServeSlot) * max_slots)) != cudaSuccess) return bad(e, "pinned allocation failed");
    if ((e = cudaMallocHost(&s->h_active, sizeof(int32_t) * max_slots)) != cudaSuccess) return bad(e, "pinned allocation failed");
    if ((e = cudaMallocHost(&s->pin_w, sizeof(int32_t) * token_budget)) != cudaSuccess) return bad(e, "pinned allocation failed");
    if ((e = cudaMallocHost(&s->pin_z, sizeof(int16_t) * token_budget)) != cudaSuccess) return bad(e, "pinned allocation failed");
    if ((e = cudaEventCreate(&s->ev0)) != cudaSuccess || (e = cudaEventCreate(&s->ev1)) != cudaSuccess)
        return bad(e, "event creation failed");
    if ((e = cudaMemset(s->d_stats, 0, sizeof(unsigned long long) * ST_TOTAL_SLOTS)) != cudaSuccess) return bad(e, "memset failed");
    std::memset(s->h_slots, 0, sizeof(ServeSlot) * max_slots);
    HandleView hv{};
    handle_view(h, &hv);
    s->tabs = hv.zargs;
    s->tabs.stats = s->d_stats;
    s->z_warps = hv.z_warps;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    s->grid = sms * serve_blocks_per_sm(hv.K, hv.z_warps);
    s->coop_grid = sms * serve_coop_blocks_per_sm(hv.K);
    if ((e = cudaGetLastError()) != cudaSuccess) return bad(e, "set-up failed");
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return PULDA_OK;
}

pulda_status pulda_serve_submit(pulda_server *s, uint64_t req_id, uint64_t seed, const int32_t *words, int32_t len,
                                int32_t n_sweeps, int16_t *z_out_host) {
    if (!s) return PULDA_ERR_INVALID;
    if (len < 1 || !words) return PULDA_ERR_INVALID;
    if (len > s->budget || len > (1 << 22)) return PULDA_ERR_INVALID;
    if (n_sweeps < 1) return PULDA_ERR_INVALID;
    const int V = s->tabs.col_ptr ? s->h->V : 0;
    for (int32_t i = 0; i < len; ++i)
        if (words[i] < 0 || words[i] >= V) return PULDA_ERR_INVALID;
    Request r;
    r.id = req_id;
    r.seed = seed;
    r.words.assign(words, words + len);
    r.n_sweeps = n_sweeps;
    r.z_out = z_out_host;
    r.submit_ns = now_ns();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->err_status != PULDA_OK) return s->err_status;
        if (s->stop) return PULDA_ERR_INVALID;
        if (s->pending.size() >= kMaxPending) return PULDA_ERR_BUSY;
        s->pending.push_back(std::move(r));
    }
    s->cv_work.notify_one();
    return PULDA_OK;
}

pulda_status pulda_serve_poll(pulda_server *s, pulda_result *out, int32_t max_results, int32_t *n_out,
                              int32_t timeout_ms) {
    if (!s || !n_out || (max_results > 0 && !out)) return PULDA_ERR_INVALID;
    *n_out = 0;
    std::unique_lock<std::mutex> lock(s->mu);
    const bool ready = s->cv_done.wait_for(lock, std::chrono::milliseconds(std::max(timeout_ms, 0)),
                                           [&] { return !s->done.empty() || s->err_status != PULDA_OK; });
    if (s->err_status != PULDA_OK && s->done.empty()) return s->err_status;
    if (!ready) return PULDA_ERR_TIMEOUT;
    int32_t n = 0;
    while (n < max_results && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = n;
    return PULDA_OK;
}

pulda_status pulda_serve_pending(pulda_server *s, int64_t *waiting, int64_t *running, int64_t *launches) {
    if (!s) return PULDA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    if (waiting) *waiting = static_cast<int64_t>(s->pending.size());
    if (running) *running = static_cast<int64_t>(s->max_slots - s->free_slots.size());
    if (launches) *launches = s->ctr[0];
    return PULDA_OK;
}

pulda_status pulda_serve_stats(pulda_server *s, int64_t *out) {
    if (!s || !out) return PULDA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    out[0] = s->ctr[0];
    out[1] = s->ctr[2];
    out[2] = s->ctr[3];
    out[3] = s->ctr[4];
    out[4] = s->ctr[5];
    out[5] = s->ctr[6];
    out[6] = static_cast<int64_t>(s->pending.size());
    out[7] = static_cast<int64_t>(s->max_slots - s->free_slots.size());
    return PULDA_OK;
}

pulda_status pulda_serve_close(pulda_server *s) {
    if (!s) return PULDA_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    pulda_status st = s->err_status;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->stream2) cudaStreamSynchronize(s->stream2);
    const pulda_options &o = s->h->opt;
    dev_free(o, s->stream, s->arena_w, false);
    dev_free(o, s->stream, s->arena_z, false);
    dev_free(o, s->stream, s->d_slots, false);
    dev_free(o, s->stream, s->d_active, false);
    dev_free(o, s->stream, s->d_work, false);
    dev_free(o, s->stream, s->d_stats, false);
    if (s->h_slots) cudaFreeHost(s->h_slots);
    if (s->h_new) cudaFreeHost(s->h_new);
    if (s->h_active) cudaFreeHost(s->h_active);
    if (s->pin_w) cudaFreeHost(s->pin_w);
    if (s->pin_z) cudaFreeHost(s->pin_z);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->stream2) cudaStreamDestroy(s->stream2);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return st;
}

}  // extern "C"
