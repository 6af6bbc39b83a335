// Many independent chains (corpora of uneven D, N, K, V) advanced together:
// every kernel of a sweep runs once over all chains' work items, and a sweep
// (six launches, or one persistent launch) is captured once into a CUDA graph
// and replayed.  The z-step CTA size, the launch form and then the alias
// tables' layout are picked by timing the candidates on the first sweeps
// (none of them changes a result, so tuning costs no extra sweeps); the
// longest documents go to the cooperative z-step by the single-chain rule.
#include <algorithm>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/pulda.h"
#include "handle.h"
#include "pulda_internal.h"

using namespace pulda;

struct pulda_batch {
    std::string err;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    pulda_options opt{};            // the caller's options (device allocator among them)
    std::vector<pulda_handle *> ch;
    std::vector<void *> allocs;
    BatchLaunch bl{};
    int sms = 1;
    int64_t sweep = 0;
    // tuning candidates (z-step warps per CTA, cooperative threshold; 0 = none),
    // timed on real sweeps: first the CTA sizes, then thresholds at the best size
    // The candidates are timed twice, in order and then in reverse, so the
    // falling cost of the first sweeps after the uniform start does not favour
    // the candidates timed later.
    struct Cand { int warps; int64_t coop_len; bool one_launch; bool packed; };
    std::vector<Cand> cand;
    std::vector<float> cand_ms;     // summed over the candidate's timed sweeps
    std::vector<int> sched;         // candidate indices still to time in this phase
    size_t sched_pos = 0;
    int phase_first = 0;            // first candidate index of the current phase
    bool tuned = false;
    // the alias layout is timed after the launch form: the best form with the
    // threshold and topic arrays, then with the packed slots
    bool tune_layout = false, layout_phase = false;
    bool one_launch = false;        // in use: one persistent launch per sweep
    bool packed = false;            // in use: the chains' tables carry packed alias slots
    std::vector<PhiArgs> hp;        // the chains' descriptors (host copies of phi / z below)
    std::vector<ZArgs> hz;
    PhiArgs *d_phi = nullptr;
    ZArgs *d_z = nullptr;
    int64_t coop_len = 0;           // in use
    std::vector<int64_t> dlen;      // document lengths in work-list order (longest first)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

pulda_status bfail(pulda_batch *b, pulda_status s, const std::string &msg) {
    if (b) b->err = msg;
    return s;
}

#define BCU(b, expr)                                                                                \
    do {                                                                                            \
        cudaError_t e_ = (expr);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? PULDA_ERR_OOM : PULDA_ERR_CUDA,     \
                         std::string(#expr " failed: ") + cudaGetErrorString(e_));                  \
    } while (0)

template <typename T>
cudaError_t balloc(pulda_batch *b, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = dev_alloc(b->opt, b->stream, sizeof(T) * std::max<size_t>(n, 1), &q, false);
    if (e == cudaSuccess) b->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return e;
}

thread_local std::string g_batch_init_error;

// Documents the cooperative z-step takes at threshold L (the work list is longest first).
int count_coop_items(const pulda_batch *b, int64_t L) {
    if (L <= 0) return 0;
    int n = 0;
    while (n < static_cast<int>(b->dlen.size()) && b->dlen[n] >= L) ++n;
    return n;
}

// Starts a tuning phase over candidates [first, cand.size()): forward, then backward.
void schedule_phase(pulda_batch *b, int first) {
    b->phase_first = first;
    b->sched.clear();
    b->sched_pos = 0;
    const int n = static_cast<int>(b->cand.size());
    for (int c = first; c < n; ++c) b->sched.push_back(c);
    for (int c = n - 1; c >= first; --c) b->sched.push_back(c);
    b->cand_ms.resize(b->cand.size(), 0.0f);
}

// Puts candidate c in use.  A change of alias layout rewrites the chains'
// descriptors on the stream, before the next sweep's launches: a sweep's
// Phi-step writes the packed slots when its descriptor has them, and its
// z-step reads whichever layout its own descriptor names.
cudaError_t apply_candidate(pulda_batch *b, const pulda_batch::Cand &c) {
    b->bl.z_warps = c.warps;
    b->bl.z_grid = b->sms * batch_z_blocks_per_sm(b->bl.kmax, c.warps, b->bl.narrow != 0);
    b->coop_len = c.coop_len;
    b->bl.n_coop = count_coop_items(b, c.coop_len);
    b->one_launch = c.one_launch;
    if (c.packed == b->packed) return cudaSuccess;
    for (size_t i = 0; i < b->ch.size(); ++i) {
        b->hp[i].apack = c.packed ? b->ch[i]->apack : nullptr;
        b->hz[i].apack = c.packed ? b->ch[i]->apack : nullptr;
    }
    const size_t n = b->ch.size();
    cudaError_t e = cudaMemcpyAsync(b->d_phi, b->hp.data(), sizeof(PhiArgs) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_z, b->hz.data(), sizeof(ZArgs) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // the host copies may change again
    if (e == cudaSuccess) b->packed = c.packed;
    return e;
}

pulda_status launch_one_sweep(pulda_batch *b) {
    if (b->one_launch) {
        BCU(b, launch_batch_sweep_persistent(b->bl, b->stream));
    } else {
        launch_batch_sweep(b->bl, b->stream);
    }
    BCU(b, cudaGetLastError());
    return PULDA_OK;
}

}  // namespace

extern "C" {

pulda_status pulda_batch_init(pulda_batch **out, const pulda_chain_desc *chains, int32_t n_chains,
                              const pulda_options *opt) {
    if (!out) return PULDA_ERR_INVALID;
    *out = nullptr;
    g_batch_init_error.clear();
    if (!chains || n_chains < 1) {
        g_batch_init_error = "n_chains must be >= 1 and chains non-NULL";
        return PULDA_ERR_INVALID;
    }
    pulda_batch *b = new pulda_batch();
    auto bail = [&](pulda_status s) {
        g_batch_init_error = b->err;
        pulda_batch_free(b);
        return s;
    };
    pulda_options o{};
    if (opt) o = *opt;
    if ((o.alloc == nullptr) != (o.free == nullptr)) {
        b->err = "alloc and free must be set together";
        return bail(PULDA_ERR_INVALID);
    }
    b->opt = o;
    if (o.docs_per_warp == 4) {
        b->err = "batched chains run one document per warp (docs_per_warp must be 0 or 1)";
        return bail(PULDA_ERR_INVALID);
    }
    if (o.phi_mode != 0) {
        b->err = "batched chains draw the Polya-urn Phi (phi_mode must be 0)";
        return bail(PULDA_ERR_INVALID);
    }
    if (o.count_path != 0) {
        b->err = "batched chains rebuild their counts by histogram (count_path must be 0)";
        return bail(PULDA_ERR_INVALID);
    }
    if (o.slice_len != 0) {
        b->err = "batched chains resample every document in order (slice_len must be 0)";
        return bail(PULDA_ERR_INVALID);
    }
    if (o.coop_min_len < -1) {
        b->err = "coop_min_len must be -1 (never), 0 (tuned) or a length";
        return bail(PULDA_ERR_INVALID);
    }
    if (o.batch_form < 0 || o.batch_form > 2 || (o.batch_form == 2 && o.coop_min_len > 0)) {
        b->err = "batch_form must be 0 (tuned), 1 (six launches) or 2 (one launch, without coop_min_len > 0)";
        return bail(PULDA_ERR_INVALID);
    }
    if (o.alias_layout < 0 || o.alias_layout > 2) {
        b->err = "alias_layout must be 0 (tuned), 1 (threshold and topic arrays) or 2 (packed slots)";
        return bail(PULDA_ERR_INVALID);
    }
    if (o.warps_per_block < 0 || o.warps_per_block > kMultiWarps) {
        b->err = "warps_per_block must be in [0, " + std::to_string(kMultiWarps) + "] (got " +
                 std::to_string(o.warps_per_block) + ")";
        return bail(PULDA_ERR_INVALID);
    }
    if (o.stream) {
        b->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            b->err = "cudaStreamCreate failed";
            return bail(PULDA_ERR_CUDA);
        }
        b->own_stream = true;
    }
    o.stream = b->stream;
    o.docs_per_warp = 1;
    // the chains' own z-step launch shape is not used: the batch launches its
    // own kernel, whose CTA size is o.warps_per_block or tuned
    pulda_options oc = o;
    oc.warps_per_block = 0;
    oc.coop_min_len = -1;
    oc.alias_layout = o.alias_layout == 1 ? 1 : 2;     // the packed slots whenever they may be used
    for (int32_t c = 0; c < n_chains; ++c) {
        const pulda_chain_desc &d = chains[c];
        pulda_handle *h = nullptr;
        pulda_status s = pulda_init(&h, d.word_ids_host, d.doc_offsets_host, d.D, d.K, d.V, d.alpha_host, d.beta,
                                    d.seed, &oc);
        if (s != PULDA_OK) {
            b->err = "chain " + std::to_string(c) + ": " + pulda_last_error(nullptr);
            return bail(s);
        }
        b->ch.push_back(h);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    // per-chain descriptors, reading the sweep counter from device memory
    GridBarrier *d_bar = nullptr;
    uint32_t *d_sweep = nullptr;
    int *d_work = nullptr;
    PhiArgs *d_phi = nullptr;
    ZArgs *d_z = nullptr;
    cudaError_t ea = cudaSuccess;
    if ((ea = balloc(b, &d_bar, 1)) != cudaSuccess || (ea = balloc(b, &d_sweep, 1)) != cudaSuccess ||
        (ea = balloc(b, &d_work, 4)) != cudaSuccess ||
        (ea = balloc(b, &d_phi, n_chains)) != cudaSuccess || (ea = balloc(b, &d_z, n_chains)) != cudaSuccess) {
        b->err = std::string("device allocation of the batch descriptors failed: ") + cudaGetErrorString(ea);
        return bail(ea == cudaErrorMemoryAllocation ? PULDA_ERR_OOM : PULDA_ERR_CUDA);
    }
    std::vector<PhiArgs> &hp = b->hp;
    std::vector<ZArgs> &hz = b->hz;
    hp.resize(n_chains);
    hz.resize(n_chains);
    b->d_phi = d_phi;
    b->d_z = d_z;
    b->packed = o.alias_layout == 2;
    std::vector<HeavyChunk> heavy;
    std::vector<std::pair<int64_t, int2>> wi, di;    // (weight, (chain, item))
    int kmax = 1;
    bool narrow = true;     // every document of every chain fits 16-bit counts
    for (int32_t c = 0; c < n_chains; ++c) {
        pulda_handle *h = b->ch[c];
        hp[c] = phi_args(h);
        hp[c].sweep_ptr = d_sweep;
        hz[c] = z_args(h, h->doc_off, h->doc_order, h->D, h->w, h->z, h->seed, 0, 0);
        hz[c].sweep_ptr = d_sweep;
        if (!b->packed) {               // the launch forms are timed with the arrays
            hp[c].apack = nullptr;
            hz[c].apack = nullptr;
        }
        kmax = std::max(kmax, h->K);
        narrow = narrow && h->narrow_all;
        for (HeavyChunk hc : h->heavy_chunks) {
            hc.chain = c;
            heavy.push_back(hc);
        }
        std::vector<int64_t> woff(h->V + 1);
        if (cudaMemcpy(woff.data(), h->word_off, sizeof(int64_t) * (h->V + 1), cudaMemcpyDeviceToHost) != cudaSuccess) {
            b->err = "reading word offsets failed";
            return bail(PULDA_ERR_CUDA);
        }
        for (int v = 0; v < h->V; ++v) wi.push_back({woff[v + 1] - woff[v], make_int2(c, v)});
        const int64_t *off = chains[c].doc_offsets_host;
        for (int64_t d = 0; d < h->D; ++d) di.push_back({off[d + 1] - off[d], make_int2(c, static_cast<int>(d))});
    }
    auto heavy_first = [](const std::pair<int64_t, int2> &x, const std::pair<int64_t, int2> &y) {
        return x.first > y.first;
    };
    std::stable_sort(wi.begin(), wi.end(), heavy_first);
    std::stable_sort(di.begin(), di.end(), heavy_first);
    std::vector<int2> wlist(wi.size()), dlist(di.size());
    for (size_t i = 0; i < wi.size(); ++i) wlist[i] = wi[i].second;
    for (size_t i = 0; i < di.size(); ++i) dlist[i] = di[i].second;
    b->dlen.resize(di.size());
    int64_t n_tokens = 0;
    for (size_t i = 0; i < di.size(); ++i) {
        b->dlen[i] = di[i].first;
        n_tokens += di[i].first;
    }
    int2 *d_wl = nullptr, *d_dl = nullptr;
    HeavyChunk *d_heavy = nullptr;
    if ((ea = balloc(b, &d_wl, wlist.size())) != cudaSuccess || (ea = balloc(b, &d_dl, dlist.size())) != cudaSuccess ||
        (ea = balloc(b, &d_heavy, heavy.size())) != cudaSuccess) {
        b->err = std::string("device allocation of the work lists failed: ") + cudaGetErrorString(ea);
        return bail(ea == cudaErrorMemoryAllocation ? PULDA_ERR_OOM : PULDA_ERR_CUDA);
    }
    cudaStream_t st = b->stream;
    const uint32_t zero = 0;
    if (cudaMemcpyAsync(d_phi, hp.data(), sizeof(PhiArgs) * n_chains, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_z, hz.data(), sizeof(ZArgs) * n_chains, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_wl, wlist.data(), sizeof(int2) * wlist.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_dl, dlist.data(), sizeof(int2) * dlist.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_sweep, &zero, sizeof zero, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(d_bar, 0, sizeof(GridBarrier), st) != cudaSuccess ||
        (!heavy.empty() && cudaMemcpyAsync(d_heavy, heavy.data(), sizeof(HeavyChunk) * heavy.size(),
                                           cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        b->err = "uploading the batch descriptors failed";
        return bail(PULDA_ERR_CUDA);
    }
    BatchLaunch &bl = b->bl;
    bl.phi = d_phi;
    bl.z = d_z;
    bl.heavy = d_heavy;
    bl.n_heavy = static_cast<int>(heavy.size());
    bl.n_chains = n_chains;
    bl.phi_items = d_wl;
    bl.n_phi_items = static_cast<int>(wlist.size());
    bl.z_items = d_dl;
    bl.n_z_items = static_cast<int>(dlist.size());
    bl.sweep = d_sweep;
    bl.work = d_work;
    bl.kmax = kmax;
    bl.narrow = narrow ? 1 : 0;
    bl.phi_grid = b->sms * batch_phi_blocks_per_sm(kmax);
    bl.coop_grid = b->sms * batch_coop_blocks_per_sm(kmax);
    bl.bar = d_bar;
    bl.persist_grid = b->sms * batch_persistent_blocks_per_sm(kmax, narrow);
    // The cooperative threshold: fixed, none, or the automatic rule of the
    // single-chain z-step over all chains' tokens (documents that would outlast
    // the pass on one warp).  It is not timed: on the 32-chain workload, timing
    // thresholds on a few sweeps chose a quarter of the rule's (and once none),
    // while over the steady sweeps the rule's threshold ran at 42.9 ms per sweep
    // against 47.2 (a quarter) and 53.0 (none).
    int64_t fixed_coop = o.coop_min_len > 0 ? o.coop_min_len : 0;
    if (o.coop_min_len == 0) {
        const int64_t L = std::max<int64_t>(kCoopAutoMin, n_tokens / kCoopAutoDiv + 1);
        if (count_coop_items(b, L) > 0) fixed_coop = L;
    }
    // Launch forms: six launches per sweep with a CTA size for the z-step, and
    // (without cooperative CTAs) one persistent launch; tuned forms are timed.
    const bool one_ok = bl.persist_grid > 0 && fixed_coop == 0;
    const bool pk = b->packed;
    if (o.batch_form == 2) {
        if (!one_ok) {
            b->err = "the one-launch form needs no document on cooperative CTAs and a resident grid";
            return bail(PULDA_ERR_INVALID);
        }
        b->cand.push_back({kMultiWarps, 0, true, pk});
    } else if (o.warps_per_block > 0) {
        b->cand.push_back({o.warps_per_block, fixed_coop, false, pk});
    } else {
        for (int w : {2, 4, 8})
            if (w <= kMultiWarps && z_step_smem(kmax, w) <= 160 * 1024) b->cand.push_back({w, fixed_coop, false, pk});
        if (b->cand.empty()) b->cand.push_back({1, fixed_coop, false, pk});
    }
    if (o.batch_form == 0 && o.warps_per_block == 0 && one_ok) b->cand.push_back({kMultiWarps, 0, true, pk});
    b->tune_layout = o.alias_layout == 0;
    if (b->cand.size() == 1 && b->tune_layout) {
        // one launch form: time the two layouts only
        pulda_batch::Cand c = b->cand.front();
        c.packed = true;
        b->cand.push_back(c);
        b->layout_phase = true;
    }
    if (b->cand.size() == 1) b->tuned = true;
    else schedule_phase(b, 0);
    if (apply_candidate(b, b->cand.front()) != cudaSuccess) {
        b->err = "uploading the batch descriptors failed";
        return bail(PULDA_ERR_CUDA);
    }
    if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess ||
        cudaStreamCreateWithFlags(&bl.stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&bl.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&bl.ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess) {
        b->err = "CUDA set-up of the batch failed";
        return bail(PULDA_ERR_CUDA);
    }
    *out = b;
    return PULDA_OK;
}

pulda_status pulda_batch_sweep(pulda_batch *b, int32_t n_sweeps) {
    if (!b) return PULDA_ERR_INVALID;
    if (n_sweeps < 0) return bfail(b, PULDA_ERR_INVALID, "n_sweeps must be >= 0");
    for (int32_t s = 0; s < n_sweeps; ++s) {
        if (!b->tuned) {
            // time the next scheduled candidate on a real sweep
            const int c = b->sched[b->sched_pos];
            BCU(b, apply_candidate(b, b->cand[c]));
            BCU(b, cudaEventRecord(b->ev0, b->stream));
            pulda_status r = launch_one_sweep(b);
            if (r != PULDA_OK) return r;
            BCU(b, cudaEventRecord(b->ev1, b->stream));
            BCU(b, cudaEventSynchronize(b->ev1));
            float ms = 0;
            BCU(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
            b->cand_ms[c] += ms;
            if (++b->sched_pos == b->sched.size()) {
                int best = b->phase_first;
                for (int k = b->phase_first; k < static_cast<int>(b->cand.size()); ++k)
                    if (b->cand_ms[k] < b->cand_ms[best]) best = k;
                if (b->tune_layout && !b->layout_phase) {
                    // the best launch form again with each alias layout
                    pulda_batch::Cand c0 = b->cand[best], c1 = b->cand[best];
                    c0.packed = false;
                    c1.packed = true;
                    const int first = static_cast<int>(b->cand.size());
                    b->cand.push_back(c0);
                    b->cand.push_back(c1);
                    b->layout_phase = true;
                    schedule_phase(b, first);
                } else {
                    BCU(b, apply_candidate(b, b->cand[best]));
                    b->tuned = true;
                }
            }
        } else {
            if (!b->exec) {
                BCU(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t le = cudaSuccess;
                if (b->one_launch) le = launch_batch_sweep_persistent(b->bl, b->stream);
                else launch_batch_sweep(b->bl, b->stream);
                cudaError_t ce = cudaStreamEndCapture(b->stream, &b->graph);
                if (le != cudaSuccess) ce = le;
                if (ce != cudaSuccess) return bfail(b, PULDA_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(ce));
                BCU(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
            }
            BCU(b, cudaGraphLaunch(b->exec, b->stream));
        }
        b->sweep += 1;
    }
    for (pulda_handle *h : b->ch) {
        h->sweep = b->sweep;
        h->have_phi = h->have_phi || b->sweep > 0;
    }
    return PULDA_OK;
}

pulda_status pulda_batch_sync(pulda_batch *b) {
    if (!b) return PULDA_ERR_INVALID;
    BCU(b, cudaStreamSynchronize(b->stream));
    for (size_t c = 0; c < b->ch.size(); ++c) {
        pulda_status s = pulda_sync(b->ch[c]);
        if (s != PULDA_OK) return bfail(b, s, "chain " + std::to_string(c) + ": " + pulda_last_error(b->ch[c]));
    }
    return PULDA_OK;
}

pulda_status pulda_batch_get_z(pulda_batch *b, int32_t chain, int16_t *z_host) {
    if (!b) return PULDA_ERR_INVALID;
    if (chain < 0 || chain >= static_cast<int32_t>(b->ch.size())) return bfail(b, PULDA_ERR_INVALID, "chain out of range");
    pulda_status s = pulda_get_z(b->ch[chain], z_host);
    if (s != PULDA_OK) return bfail(b, s, pulda_last_error(b->ch[chain]));
    return PULDA_OK;
}

pulda_status pulda_batch_stats(pulda_batch *b, int32_t chain, pulda_sweep_stats *out) {
    if (!b) return PULDA_ERR_INVALID;
    if (chain < 0 || chain >= static_cast<int32_t>(b->ch.size())) return bfail(b, PULDA_ERR_INVALID, "chain out of range");
    pulda_status s = pulda_stats(b->ch[chain], out);
    if (s != PULDA_OK) return bfail(b, s, pulda_last_error(b->ch[chain]));
    return PULDA_OK;
}

pulda_status pulda_batch_tuning(pulda_batch *b, int32_t *z_warps, int32_t *coop_min_len, int32_t *tuned,
                                int32_t *one_launch, int32_t *alias_layout) {
    if (!b) return PULDA_ERR_INVALID;
    if (one_launch) *one_launch = b->one_launch ? 1 : 0;
    if (alias_layout) *alias_layout = b->packed ? 2 : 1;
    if (z_warps) *z_warps = b->one_launch ? kMultiWarps : b->bl.z_warps;
    if (coop_min_len) *coop_min_len = static_cast<int32_t>(b->coop_len > 0 ? b->coop_len : -1);
    if (tuned) *tuned = b->tuned ? 1 : 0;
    return PULDA_OK;
}

const char *pulda_batch_last_error(const pulda_batch *b) { return b ? b->err.c_str() : g_batch_init_error.c_str(); }

void pulda_batch_free(pulda_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->bl.stream2) {
        cudaStreamSynchronize(b->bl.stream2);
        cudaStreamDestroy(b->bl.stream2);
    }
    if (b->bl.ev_fork) cudaEventDestroy(b->bl.ev_fork);
    if (b->bl.ev_join) cudaEventDestroy(b->bl.ev_join);
    for (pulda_handle *h : b->ch) pulda_free(h);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (void *p : b->allocs) dev_free(b->opt, b->stream, p, false);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

pulda_status pulda_barrier_selftest(int32_t blocks, int32_t missing, int32_t rounds, int32_t *passed) {
    if (blocks < 1 || missing < 0 || rounds < 1 || !passed) return PULDA_ERR_INVALID;
    int sms = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (blocks > sms) return PULDA_ERR_INVALID;            // one 32-thread CTA per SM at most: all resident
    void *mem = nullptr;
    if (cudaMalloc(&mem, 256) != cudaSuccess) return PULDA_ERR_OOM;
    auto *bar = static_cast<GridBarrier *>(mem);
    auto *err = reinterpret_cast<unsigned long long *>(static_cast<char *>(mem) + 64);
    auto *cnt = reinterpret_cast<unsigned *>(static_cast<char *>(mem) + 128);
    pulda_status st = PULDA_OK;
    unsigned long long herr = 0;
    unsigned hcnt = 0;
    if (cudaMemset(mem, 0, 256) != cudaSuccess ||
        launch_barrier_selftest(bar, blocks, missing, rounds, err, cnt, nullptr) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&herr, err, sizeof herr, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&hcnt, cnt, sizeof hcnt, cudaMemcpyDeviceToHost) != cudaSuccess)
        st = PULDA_ERR_CUDA;
    else if (herr & ERR_BARRIER)
        st = PULDA_ERR_TIMEOUT;
    cudaFree(mem);
    *passed = static_cast<int32_t>(hcnt);
    return st;
}

}  // extern "C"
