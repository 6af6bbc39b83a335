#!/usr/bin/env python3
"""Benchmark of the Polya-urn LDA sampler on GB300.

One step = one sweep of Algorithm 2 over the whole large synthetic corpus
(D=300,000 documents, V=100,000, ~99M tokens, K=1,000): the Phi-step (counts,
Poisson draws, dead-row fix-up, column offsets, per-word tables) and the
z-step.  ``value`` is tokens per second of whole sweeps; the roofline object
reports the z-step kernel's algorithmic bytes per launch over its measured
duration against the measured HBM copy bandwidth.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pulda|reference]

Under torchrun (N > 1) every rank runs its own chain (seed = rank) on its own
GPU: the chains are independent, so there is no collective on the data path
and the scaling is weak.  ``--impl reference`` times the CPU oracle on the
host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import ctypes
import csv
import hashlib
import io
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "z-step tokens/s/GPU at K=1000 (% HBM roofline); serving p50/p99 vs plain"
K_TOPICS = 1000
ALPHA, BETA = 0.1, 0.01
def kernels_per_sweep(w: np.ndarray, phi_mode: int, layout: dict | None = None, slice_docs: int = 0) -> int:
    """Library kernels one sweep launches: the frequent-word histogram (when a
    word has more than 2^17 tokens), then Polya urn: counts+draws, dead-row
    fix-up, column scan, per-word tables; Dirichlet: counts, Gamma draws, two
    row-sum passes, selection, column scan, per-word tables; then the z-step
    as the handle laid it out (pulda_z_layout): its main kernel, the
    cooperative kernel when some document is on CTAs, the one-warp kernel for
    documents too long for four per warp, or the pass-start counts before a
    z-step in slices."""
    heavy = 1 if np.bincount(w).max(initial=0) > (1 << 17) else 0
    extra = 1 if slice_docs > 0 else 0
    if layout is not None:
        extra += (1 if layout["coop_docs"] > 0 else 0)
        if layout["docs_per_warp"] == 4:
            extra += 1 if layout["one_warp_docs"] > 0 else 0
    return heavy + (4 if phi_mode == 0 else 7) + 1 + extra


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--burnin", type=int, default=25,
                    help="untimed sweeps before the warm-up: the default times sweeps 31-50 of the "
                         "50-sweep large workload rather than the first sweeps after a uniform start")
    ap.add_argument("--impl", choices=["pulda", "reference"], default="pulda")
    ap.add_argument("--cpu-docs", type=int, default=20000, help="documents in the CPU oracle's bounded sample")
    ap.add_argument("--ref-docs", type=int, default=5000,
                    help="documents in each step of the reference (oracle) arm's bounded sample")
    ap.add_argument("--K", type=int, default=1000,
                    help="topics the sampler runs with (the corpora are drawn with K=1000 topics either way)")
    ap.add_argument("--count-path", type=int, default=0, choices=[0, 1],
                    help="Phi-step count rebuild: 0 shared-memory histograms, 1 radix sort of (word, topic) keys")
    ap.add_argument("--heaps-sizes", type=str, default="1000000,4000000,16000000,64000000",
                    help="heaps form: corpus sizes (tokens)")
    ap.add_argument("--heaps-xi", type=float, default=20.0, help="heaps form: V = xi N^psi")
    ap.add_argument("--heaps-psi", type=float, default=0.5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving keys of the sweep line")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched keys of the sweep line")
    ap.add_argument("--serve-low-requests", type=int, default=150,
                    help="serving keys: requests of the trace both arms serve at half the plain arm's capacity")
    ap.add_argument("--serve-high-rate", type=float, default=5000.0, help="serving keys: the continuous arm's high rate")
    ap.add_argument("--serve-high-seconds", type=float, default=2.0, help="serving keys: its arrival window")
    ap.add_argument("--batch-steps", type=int, default=10, help="batched keys: timed sweeps of each arm")
    ap.add_argument("--batch-form", type=int, default=0, choices=[0, 1, 2],
                    help="batched launch form: 0 tuned, 1 six launches per sweep, 2 one persistent launch")
    ap.add_argument("--alias-layout", type=int, default=0, choices=[0, 1, 2],
                    help="alias tables: 1 threshold and topic arrays, 2 packed slots, 0 = arrays for the sweep "
                         "form and tuned for the batched one")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--docs-per-warp", type=int, default=0, help="z-step documents per warp: 0 auto, 1 or 4")
    ap.add_argument("--phi-mode", type=int, default=0, choices=[0, 1],
                    help="sweep form: 0 = Polya-urn Phi (Algorithm 2), 1 = Dirichlet Phi (Algorithm 1)")
    ap.add_argument("--rates", type=str, default="2000,5000,10000,20000,50000",
                    help="serving: Poisson arrival rates, documents per second")
    ap.add_argument("--serve-seconds", type=float, default=1.5, help="serving: arrival window per rate")
    ap.add_argument("--slice", type=int, default=0,
                    help="serving: tokens a request advances per launch (0 = tuned by the server)")
    ap.add_argument("--serve-sweeps", type=int, default=50, help="serving: z-sweeps per request")
    ap.add_argument("--plain-requests", type=int, default=150,
                    help="serving: requests the one-at-a-time baseline serves (the first ones, at the lowest rate)")
    ap.add_argument("--form", choices=["sweep", "batched", "serving", "trace", "sparsity", "heaps"], default="sweep",
                    help="sweep: the large corpus (the headline line); batched: 32 uneven chains in one graph "
                         "launch per sweep against 32 sequential single-chain runs; trace: the log posterior "
                         "after every sweep, Polya urn against Dirichlet Phi, on the same corpus and seed; sparsity: "
                         "both Phi-steps timed on the large corpus pruned by vocabulary size, rare-word "
                         "threshold and data size")
    ap.add_argument("--slice-len", type=int, default=0,
                    help="sweep/trace forms: documents longer than this in stale-count slices (0 = Algorithm 2)")
    ap.add_argument("--trace-corpus", choices=["small", "large"], default="small")
    ap.add_argument("--trace-sweeps", type=int, default=100)
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="fraction of each batched chain's documents (1.0 = the full 267M-token workload)")
    ap.add_argument("--coop-min-len", type=int, default=0,
                    help="documents (serving: requests) at least this long resampled by a CTA of four warps "
                         "(0 = automatic, -1 = never); results are identical")
    ap.add_argument("--docs", type=int, default=300_000,
                    help="documents of the large corpus (300,000 = the full workload; fewer for profiling)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for r in csv.reader(f):
                if len(r) >= 9:
                    rows.append([x.strip() for x in r])
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# --------------------------------------------------------------- helpers
def peaks() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def code_hash(text: str) -> str:
    """Hash of a source's code: // comments, trailing blanks and empty lines do not count."""
    lines = []
    for line in text.splitlines():
        i = line.find("//")
        code = (line[:i] if i >= 0 else line).rstrip()
        if code:
            lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


# The sources the one-warp z-step kernel is compiled from.
Z_STEP_SOURCES = ("kernels.cu", "zstep.cuh", "device_rng.cuh", "checks.cuh", "pulda_internal.h")


def kernel_source_hash() -> str:
    text = []
    for name in Z_STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1704_03581_gb300", "csrc", name)) as f:
            text.append(f.read())
    return code_hash("\n".join(text))


def recorded_profile() -> dict:
    """The committed ncu record of one full-size z-step launch, if it was taken
    on the current kernel source, else {}."""
    p = os.path.join(ROOT, "profiles", "z_step_large_traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)
        if rec.get("source_sha") == kernel_source_hash():
            return rec
    except Exception:
        pass
    return {}


def recorded_traffic() -> float | None:
    """DRAM bytes per z-step launch from the committed ncu record, or None."""
    rec = recorded_profile()
    return float(rec["dram_bytes_per_launch"]) if "dram_bytes_per_launch" in rec else None


def count_word_topic_pairs(s, K: int, V: int) -> int:
    """nnz(n): the nonzero (word, topic) counts of the sampler's current topics,
    from the library's own count export (a diagnostic, outside any timing)."""
    import paper_1704_03581_gb300 as P
    n = np.empty(K * V, np.int32)
    P.pulda_get_counts(s.h, n, None)
    return int(np.count_nonzero(n))


def phi_bytes(N: int, nnz_phi: int, nnz_n: int) -> float:
    """Algorithmic bytes of one Phi-step with its count rebuild: each token's
    topic gathered through the word-major permutation (4 + 2 B), 14 B per
    nonzero of Phi (its draw and tables) and 8 B per nonzero of n."""
    return 6.0 * N + 14.0 * nnz_phi + 8.0 * nnz_n


def phi_roofline(ms_per_sweep: float, N: int, nnz_phi: int, nnz_n: int, peak: float) -> dict:
    b = phi_bytes(N, nnz_phi, nnz_n)
    achieved = b / (ms_per_sweep / 1000.0) / 1e9
    return {"ms_per_sweep": ms_per_sweep, "nnz_phi": nnz_phi, "nnz_n": nnz_n, "bytes_per_sweep": b,
            "bytes_model": "6 B per token + 14 B per nonzero of Phi + 8 B per nonzero of n",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak}


def issue_roofline(tokens_per_s: float, sm_mhz: float | None) -> dict | None:
    """The z-step against the SMs' instruction-issue rate: warp instructions per
    token (ncu, one full-size launch) times the measured tokens/s, against
    SMs x 4 schedulers x 1 warp instruction per cycle at the sampled SM clock."""
    rec = recorded_profile()
    if "warp_instructions_per_token" not in rec:
        return None
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_mhz or 2070.0
    peak = sms * 4 * mhz * 1e6
    achieved = float(rec["warp_instructions_per_token"]) * tokens_per_s
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak, "warp_instructions_per_token": rec["warp_instructions_per_token"],
            "peak_kind": f"{sms} SMs x 4 schedulers x 1 instruction/cycle at {mhz:.0f} MHz"}


def z_bytes(tokens: int, sum_min: int, a_branch: int, docs: int) -> int:
    """Algorithmic HBM bytes of z-steps over `tokens` tokens, a model of what
    the method must touch: per token the word id (4), its topic
    in and out (2+2) and sigma_a of its word (4); per element of the smaller
    of the document's and the word's nonzero topics one topic id and one
    weight (2+4) -- min(K_d, K_v) of them (complexity theorem); per alias draw
    one slot (threshold and topic, padded to 8); per document its offset (8)."""
    return 12 * tokens + 6 * sum_min + 8 * a_branch + 8 * docs


def z_bytes_impl(tokens: int, sum_min: int, a_branch: int, docs: int) -> int:
    """The same with this implementation's widths: sigma_a held as a 64-bit
    integer (8) and the column offset read per token (8); an alias slot 4+2."""
    return 24 * tokens + 6 * sum_min + 6 * a_branch + 8 * docs


def reduce_max(x: float, world: int, device=None) -> float:
    """Max of x over all ranks (identity on one rank).  NCCL reduces device
    tensors, gloo host tensors."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = device if device is not None else ("cuda" if dist.get_backend() == "nccl" else "cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_tokens_per_s(tokens_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank resamples its own chain of the same
    size, so the job does world x tokens x steps in the slowest rank's time."""
    return world * tokens_per_rank * steps / (ms_max / 1000.0)


def cpu_count() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------- CPU oracle
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def oracle_sample(corpus, docs: int, warm: int = 0, threads: int = 1):
    """One oracle sweep (Phi-step + z-step) over the first `docs` documents, a
    bounded sample of the same workload, on `threads` host threads (the
    threaded oracle gives the single-threaded results)."""
    from oracle import oracle as O
    sub = corpus.slice_docs(0, min(docs, corpus.D))
    ch = O.Chain(sub.w, sub.doc_off, K_TOPICS, corpus.V, ALPHA, BETA, seed=0, threads=threads)
    for _ in range(warm):
        ch.sweep(1)
    t0 = time.perf_counter()
    ch.sweep(1)
    dt = time.perf_counter() - t0
    return sub.N, dt


def run_reference(args, corpus):
    steps, warm = args.steps, args.warmup
    tot_tok, tot_t = 0, 0.0
    from oracle import oracle as O
    cores = O.host_threads()
    sub = corpus.slice_docs(0, min(args.ref_docs, corpus.D))
    ch = O.Chain(sub.w, sub.doc_off, K_TOPICS, corpus.V, ALPHA, BETA, seed=0, threads=cores)
    for _ in range(warm):
        ch.sweep(1)
    for _ in range(steps):
        t0 = time.perf_counter()
        ch.sweep(1)
        tot_t += time.perf_counter() - t0
        tot_tok += sub.N
    v = tot_tok / tot_t
    sample = (f"one oracle sweep per step over the first {sub.D} documents ({sub.N} tokens) of the large "
              f"corpus, K={K_TOPICS}, on {cores} host threads (results equal the single-threaded oracle's)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "tokens/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1000.0 * tot_t / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": corpus.name, "sample_docs": sub.D, "sample_tokens": sub.N, "K": K_TOPICS},
        "cpu_baseline": {"value": v, "unit": "tokens/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": v, "unit": "tokens/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU
def run_pulda(args, corpus, rank: int, world: int):
    import torch
    import torch.distributed as dist
    import paper_1704_03581_gb300 as P

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = P.Sampler(corpus.w, corpus.doc_off, K_TOPICS, corpus.V, ALPHA, BETA, seed=rank,
                  stream=stream.cuda_stream, docs_per_warp=args.docs_per_warp,
                  phi_mode=args.phi_mode, slice_len=args.slice_len, coop_min_len=args.coop_min_len,
                  count_path=args.count_path, alias_layout=args.alias_layout)
    layout = s.z_layout()
    s.sweep(args.burnin + args.warmup)
    s.sync()
    lp_before = s.log_posterior()[0]          # the diagnostic, outside the timed region
    st0 = s.stats()
    first_timed = st0["sweep"] + 1
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", dev)))
    clocks.start()
    e0.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        P.pulda_phi_step(s.h)
        ev[k][1].record(stream)
        P.pulda_z_step(s.h)
        ev[k][2].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    s.sync()
    ms = e0.elapsed_time(e1)
    phi_ms = sum(ev[k][0].elapsed_time(ev[k][1]) for k in range(K))
    z_ms = sum(ev[k][1].elapsed_time(ev[k][2]) for k in range(K))
    st1 = s.stats()
    ms_max = reduce_max(ms, world)
    if world > 1:
        dist.barrier()
    tokens = st1["cum_tokens"] - st0["cum_tokens"]
    sum_min = st1["cum_sum_min"] - st0["cum_sum_min"]
    a_br = st1["cum_a_branch"] - st0["cum_a_branch"]
    sum_int = st1["cum_sum_inter"] - st0["cum_sum_inter"]
    docside = st1["cum_docside"] - st0["cum_docside"]
    assert tokens == K * corpus.N, (tokens, K * corpus.N)
    nnz_phi = st1["nnz_phi"]
    nnz_n = count_word_topic_pairs(s, K_TOPICS, corpus.V)   # for the Phi-step's byte model, not timed
    torch.cuda.synchronize()
    t_lp = time.perf_counter()
    lp_after = s.log_posterior()[0]
    lp_ms = 1000.0 * (time.perf_counter() - t_lp)
    serving = None
    if world == 1 and not args.no_serving:
        # fold-in serving against this chain's Phi after its sweeps (not timed above)
        serving = serving_probe(s, corpus.V, args.serve_sweeps, args.slice, args.serve_low_requests,
                                args.serve_high_rate, args.serve_high_seconds)
    s.close()

    e2e = None
    if not args.no_e2e:
        # the public API end to end: host corpus in, sweeps, host topics out
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = P.Sampler(corpus.w, corpus.doc_off, K_TOPICS, corpus.V, ALPHA, BETA, seed=rank,
                       stream=stream.cuda_stream, docs_per_warp=args.docs_per_warp, phi_mode=args.phi_mode,
                       slice_len=args.slice_len, coop_min_len=args.coop_min_len, alias_layout=args.alias_layout)
        s2.sync()
        t_init = time.perf_counter() - t0
        stats_bytes = ctypes.sizeof(P.SweepStats)
        for _ in range(K):
            s2.sweep(1)
            s2.stats()      # the sweep's counters read back to the host (its result)
        zh = s2.z()         # e2e covers sweeps 1..K from the uniform start
        dt = time.perf_counter() - t0
        s2.close()
        h2d = corpus.w.nbytes + corpus.doc_off.nbytes + 4 * K_TOPICS
        d2h = zh.nbytes + K * stats_bytes
        dt_max = reduce_max(dt, world)
        e2e = {"value": aggregate_tokens_per_s(corpus.N, K, world, 1000.0 * dt_max), "unit": "tokens/s",
               "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
               "init_ms": 1000.0 * t_init,
               "note": "pulda_init from host buffers (the corpus crosses once: every sweep reads it on the "
                       "device), then per sweep the sweep and a read of its counters to the host, then the "
                       "topics to the host; host clock"}

    batched = None
    if world == 1 and not args.no_batched:
        batched = batched_probe(args.batch_scale, args.batch_steps, 12, args.coop_min_len, batch_form=args.batch_form,
                                alias_layout=args.alias_layout)
    if rank != 0:
        return
    peak, peak_kind = peaks()
    zbytes = z_bytes(tokens, sum_min, a_br, K * corpus.D)
    achieved = zbytes / K / (z_ms / K / 1000.0) / 1e9
    achieved_impl = z_bytes_impl(tokens, sum_min, a_br, K * corpus.D) / K / (z_ms / K / 1000.0) / 1e9
    traffic = recorded_traffic()
    cpu = None
    if world == 1 and not args.no_cpu:
        from oracle import oracle as O
        cores = O.host_threads()
        n_tok, dt = oracle_sample(corpus, args.cpu_docs, threads=cores)
        n1, dt1 = oracle_sample(corpus, args.cpu_docs, threads=1)
        cpu = {"value": n_tok / dt, "unit": "tokens/s", "cores": cores, "kind": "oracle",
               "cpu_model": cpu_model(),
               "sample": f"one oracle sweep (Phi-step + z-step) over the first {min(args.cpu_docs, corpus.D)} "
                         f"documents ({n_tok} tokens) of the same corpus, K={K_TOPICS}, on {cores} host threads "
                         f"(words and documents split over the threads; results equal the single-threaded "
                         f"oracle's)",
               "single_core": {"value": n1 / dt1, "unit": "tokens/s", "cores": 1}}
    line = {
        "metric": METRIC,
        "value": aggregate_tokens_per_s(corpus.N, K, world, ms_max),
        "unit": "tokens/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": ms_max / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int64",
        "data": "synthetic (LDA generative process, Zipf(1.05) vocabulary)",
        "config": {"workload": corpus.name, "D": corpus.D, "V": corpus.V, "N": corpus.N, "K": K_TOPICS,
                   "alpha": ALPHA, "beta": BETA, "parallelism": f"{world} independent chains (replicas)",
                   "l2": (f"inputs {'larger' if 6 * corpus.N > 129e6 else 'smaller'} than L2 (word ids "
                          f"{4 * corpus.N / 1e6:.0f} MB + topics {2 * corpus.N / 1e6:.0f} MB read every sweep)"),
                   "timed_sweeps": [first_timed, first_timed + K - 1],
                   "phi": "Dirichlet (Algorithm 1)" if args.phi_mode == 1 else "Poisson Polya urn (Algorithm 2)",
                   "z": (f"documents over {args.slice_len} tokens in stale-count slices (not the paper's sampler)"
                         if args.slice_len > 0 else "every document in order (Algorithm 2)"),
                   "alias": "packed 8-byte slots" if args.alias_layout == 2 else "threshold and topic arrays"},
        "z_step": {"tokens_per_s": K * corpus.N / (z_ms / 1000.0), "ms_per_launch": z_ms / K,
                   "mean_min_kd_kv": sum_min / tokens, "mean_intersection": sum_int / tokens,
                   "docside_frac": docside / tokens, "a_branch_frac": a_br / tokens},
        "phi_step": phi_roofline(phi_ms / K, corpus.N, nnz_phi, nnz_n, peak),
        "sweep_roofline": {"bytes_per_sweep": zbytes / K + phi_bytes(corpus.N, nnz_phi, nnz_n),
                           "achieved": (zbytes / K + phi_bytes(corpus.N, nnz_phi, nnz_n)) / (ms_max / K / 1000.0) / 1e9,
                           "peak": peak, "unit": "GB/s",
                           "frac": (zbytes / K + phi_bytes(corpus.N, nnz_phi, nnz_n)) / (ms_max / K / 1000.0) / 1e9 / peak,
                           "bytes_model": "the z-step's and the Phi-step's algorithmic bytes over the whole sweep"},
        "log_posterior": {"before_timed": lp_before, "after_timed": lp_after, "ms_per_evaluation": lp_ms,
                          "note": "collapsed log p(w, z | alpha, beta), not timed"},
        "roofline_issue": issue_roofline(K * corpus.N / (z_ms / 1000.0), (clk or {}).get("sm_mhz")),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_z_step" if layout["docs_per_warp"] == 1 else "k_z_step_grouped",
                     "peak_kind": f"{peak_kind} HBM copy bandwidth",
                     "algorithmic_bytes_per_launch": zbytes / K,
                     "bytes_model": "12 B per token + 6 B per min(K_d, K_v) element + 8 B per alias draw + "
                                    "8 B per document",
                     "frac_implementation_bytes": achieved_impl / peak,
                     "implementation_bytes_model": "24 B per token (64-bit sigma_a, column offset) + 6 B per "
                                                   "min(K_d, K_v) element + 6 B per alias draw + 8 B per document"},
        "gpu_launches": kernels_per_sweep(corpus.w, args.phi_mode, layout,
                                          int(args.slice_len > 0 and np.diff(corpus.doc_off).max() > args.slice_len)) * K,
        "z_kernel": (f"{'four documents' if layout['docs_per_warp'] == 4 else 'one document'} per warp; "
                     f"{layout['coop_docs']} longest documents on one CTA each"),
        "clocks": clk,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "serving": serving,
        "batched": batched,
    }
    print(json.dumps(line), flush=True)


def run_trace(args):
    """The paper's mixing comparison (Section 5, log-posterior per iteration) and
    its Phi-step comparison: the same corpus and seed run under the Polya-urn
    Phi (Algorithm 2) and the Dirichlet Phi (Algorithm 1), the collapsed log
    p(w, z) recorded after every sweep (not timed) and each half-step timed
    with CUDA events."""
    import torch
    import paper_1704_03581_gb300 as P
    from paper_1704_03581_gb300 import synth

    if args.trace_corpus == "small":
        corpus, K = synth.small(), 100
    else:
        corpus, K = synth.large(D=args.docs), K_TOPICS
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {}
    if args.slice_len > 0:      # Algorithm 2 against its stale-count slices
        runs = ((0, 0, "algorithm_2"), (0, args.slice_len, "slices"))
    else:                       # the Polya urn against Algorithm 1's Dirichlet Phi
        runs = ((0, 0, "polya_urn"), (1, 0, "dirichlet"))
    for mode, sl, name in runs:
        s = P.Sampler(corpus.w, corpus.doc_off, K, corpus.V, ALPHA, BETA, seed=0, stream=stream.cuda_stream,
                      phi_mode=mode, slice_len=sl)
        lp, phi_ms, z_ms, nnz = [float(s.log_posterior()[0])], [], [], []
        for _ in range(args.trace_sweeps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            P.pulda_phi_step(s.h)
            e[1].record(stream)
            P.pulda_z_step(s.h)
            e[2].record(stream)
            lp.append(float(s.log_posterior()[0]))       # synchronises
            phi_ms.append(e[0].elapsed_time(e[1]))
            z_ms.append(e[1].elapsed_time(e[2]))
            nnz.append(s.stats()["nnz_phi"])
        s.close()
        tail = max(1, args.trace_sweeps // 5)
        out[name] = {"log_posterior": lp, "phi_ms": float(np.median(phi_ms)), "z_ms": float(np.median(z_ms)),
                     "nnz_phi_last": int(nnz[-1]), "mean_last_fifth": float(np.mean(lp[-tail:]))}
    na, nb = runs[0][2], runs[1][2]
    a, b = out[na], out[nb]
    line = {
        "metric": ("log-posterior trace per sweep: Algorithm 2 vs stale-count slices of "
                   f"{args.slice_len} tokens" if args.slice_len > 0 else
                   "log-posterior trace per sweep: Polya urn (Algorithm 2) vs Dirichlet (Algorithm 1)"),
        "value": (a["mean_last_fifth"] - b["mean_last_fifth"]) / abs(b["mean_last_fifth"]),
        "unit": "relative difference of the mean log posterior over the last fifth of the sweeps",
        "n_gpus": 1, "steps": args.trace_sweeps, "higher_is_better": False, "dtype": "int64",
        "data": "synthetic (LDA generative process)",
        "config": {"workload": corpus.name, "D": corpus.D, "V": corpus.V, "N": corpus.N, "K": K,
                   "alpha": ALPHA, "beta": BETA, "seed": 0},
        "phi_step_ms": {na: a["phi_ms"], nb: b["phi_ms"], "ratio": b["phi_ms"] / a["phi_ms"]},
        "z_step_ms": {na: a["z_ms"], nb: b["z_ms"], "ratio": b["z_ms"] / a["z_ms"]},
        "nnz_phi_last": {na: a["nnz_phi_last"], nb: b["nnz_phi_last"]},
        "traces": {na: a["log_posterior"], nb: b["log_posterior"]},
    }
    print(json.dumps(line), flush=True)


def run_sparsity(args):
    """The paper's runtime study over vocabulary sizes, rare-word thresholds and
    data sizes (Section 5, the figure on sparsity): the large corpus pruned to
    its top-TF-IDF words, with its rare words removed, or cut to its first
    documents, each sampled from the same seed under the Polya-urn Phi
    (Algorithm 2) and the Dirichlet Phi (Algorithm 1).  After ``--burnin``
    sweeps the Phi- and z-steps of the next ``--steps`` sweeps are timed with
    CUDA events on the sampler's stream."""
    import torch
    import paper_1704_03581_gb300 as P
    from paper_1704_03581_gb300 import synth

    base = synth.large(D=args.docs)
    scores = synth.tfidf(base)
    cases = [("vocabulary", base.V, base)]
    cases += [("vocabulary", v, synth.tfidf_pruned(base, v, scores)) for v in (50_000, 20_000, 5_000)]
    cases += [("rare_threshold", t, synth.rare_word_pruned(base, t)) for t in (50, 200, 1000)]
    cases += [("documents", d, base.slice_docs(0, d)) for d in (base.D // 8, base.D // 4, base.D // 2)]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def measure(c, mode):
        s = P.Sampler(c.w, c.doc_off, K_TOPICS, c.V, ALPHA, BETA, seed=0, stream=stream.cuda_stream, phi_mode=mode)
        s.sweep(args.burnin)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        mins = []
        for e in ev:
            e[0].record(stream)
            P.pulda_phi_step(s.h)
            e[1].record(stream)
            P.pulda_z_step(s.h)
            e[2].record(stream)
            st = s.stats()                                   # synchronises; outside the events
            mins.append(st["sum_min"] / max(1, st["tokens"]))
        phi = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
        z = float(np.median([e[1].elapsed_time(e[2]) for e in ev]))
        out = {"phi_ms": phi, "z_ms": z, "sweep_ms": phi + z, "nnz_phi": int(st["nnz_phi"]),
               "mean_min_kd_kv": float(np.mean(mins))}
        s.close()
        return out

    rows = []
    for axis, setting, c in cases:
        a, b = measure(c, 0), measure(c, 1)
        rows.append({"axis": axis, "setting": setting, "V": c.V, "D": c.D, "N": c.N, "polya_urn": a, "dirichlet": b,
                     "ratio_sweep": b["sweep_ms"] / a["sweep_ms"], "ratio_z": b["z_ms"] / a["z_ms"],
                     "ratio_phi": b["phi_ms"] / a["phi_ms"]})
        print(json.dumps({"progress": f"{axis}={setting}", "ratio_sweep": rows[-1]["ratio_sweep"]}),
              file=sys.stderr, flush=True)
    full = rows[0]
    line = {
        "metric": "sweep time vs vocabulary size, rare-word threshold and data size: Dirichlet Phi (Algorithm 1) "
                  "over Polya urn (Algorithm 2)",
        "value": full["ratio_sweep"],
        "unit": "ratio of median sweep times (Dirichlet / Polya urn) on the unpruned corpus",
        "n_gpus": 1, "steps": args.steps, "warmup": args.burnin, "higher_is_better": True, "dtype": "int64",
        "data": "synthetic (LDA generative process, Zipf(1.05) vocabulary), pruned on the host",
        "config": {"workload": base.name, "K": K_TOPICS, "alpha": ALPHA, "beta": BETA, "seed": 0,
                   "vocabulary": "top words by corpus TF-IDF (count x ln(D/df))",
                   "rare_threshold": "words with fewer occurrences removed",
                   "documents": "the first D documents"},
        "rows": rows,
    }
    print(json.dumps(line), flush=True)


def batched_probe(scale: float, steps: int, warmup: int, coop_min_len: int, clocks_too: bool = False,
                  batch_form: int = 0, alias_layout: int = 0) -> dict:
    """32 independent corpora (uneven D, N, K, V; D scaled by `scale`) advanced
    together by one CUDA-graph launch per sweep, against the same 32 chains
    run one after another through single-chain handles (each with its own
    best launch layout); both must give identical topics.  Sweeps 1..warmup
    (the batch times its tuning candidates there) are not timed."""
    import torch
    import paper_1704_03581_gb300 as P
    from paper_1704_03581_gb300 import synth

    t_gen = time.monotonic()
    specs = synth.batched_specs(32)
    corpora = synth.batched_corpora(specs, scale)
    t_gen = time.monotonic() - t_gen
    chains = [dict(w=c.w, doc_off=c.doc_off, K=sp["K"], V=sp["V"], alpha=ALPHA, beta=BETA, seed=sp["seed"])
              for c, sp in zip(corpora, specs)]
    N = sum(c.N for c in corpora)
    stream = torch.cuda.Stream()
    K, W = steps, max(warmup, 12)
    b = P.Batch(chains, stream=stream.cuda_stream, coop_min_len=coop_min_len, batch_form=batch_form,
                alias_layout=alias_layout)
    b.sweep(W)                          # the first sweeps also time the tuning candidates
    b.sync()
    assert b.tuning()[2], "tuning not over after the warm-up sweeps"
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device()) if clocks_too else None
    if clocks:
        clocks.start()
    e0.record(stream)
    b.sweep(K)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    b.sync()
    ms_b = e0.elapsed_time(e1)
    zb = [b.z(i) for i in range(len(chains))]
    warps, coop_len, _, one_launch, layout = b.tuning()
    b.close()
    del b
    # the same chains, one after another, one handle each
    same = True
    ms_s = 0.0
    for i, c in enumerate(chains):
        s1 = P.Sampler(c["w"], c["doc_off"], c["K"], c["V"], c["alpha"], c["beta"], c["seed"],
                       stream=stream.cuda_stream)
        s1.sweep(W)
        torch.cuda.synchronize()
        e0.record(stream)
        s1.sweep(K)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_s += e0.elapsed_time(e1)
        same &= bool(np.array_equal(zb[i], s1.z()))
        s1.close()
    return {"workload": f"32 chains, D log-uniform [1e3, 1e5] scaled by {scale}, mean length log-uniform "
                        f"[50, 2000], V log-uniform [5e3, 5e4], K in {{50, 100, 200, 500}}",
            "N": N, "timed_sweeps": [W + 1, W + K], "tokens_per_s": N * K / (ms_b / 1000.0),
            "ms_per_sweep": ms_b / K, "sequential_tokens_per_s": N * K / (ms_s / 1000.0),
            "sequential_ms_per_sweep": ms_s / K, "speedup_vs_sequential": ms_s / ms_b,
            "identical_topics": same, "z_warps_tuned": warps, "coop_min_len_tuned": coop_len,
            "alias_layout": "packed 8-byte slots" if layout == 2 else "threshold and topic arrays",
            "launch_form": "one persistent launch per sweep" if one_launch else "six launches per sweep (a graph)",
            "gpu_launches": (1 if one_launch else 6 + (1 if coop_len > 0 else 0)) * K, "generation_s": t_gen,
            "clocks": clk}


def run_batched(args):
    """The batched-chains form alone (config 4)."""
    r = batched_probe(args.batch_scale, args.steps, args.warmup, args.coop_min_len, clocks_too=True,
                      batch_form=args.batch_form, alias_layout=args.alias_layout)
    line = {
        "metric": "batched chains: tokens/s of 32 uneven chains in one graph launch per sweep vs 32 sequential "
                  "single-chain runs",
        "value": r["tokens_per_s"], "unit": "tokens/s", "n_gpus": 1, "steps": args.steps, "warmup": r["timed_sweeps"][0] - 1,
        "ms_per_step": r["ms_per_sweep"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": r["workload"], "N": r["N"], "z_warps_tuned": r["z_warps_tuned"],
                   "coop_min_len_tuned": r["coop_min_len_tuned"], "alias_layout": r["alias_layout"],
                   "launch_form": r["launch_form"]},
        "sequential": {"value": r["sequential_tokens_per_s"], "ms_per_step": r["sequential_ms_per_sweep"]},
        "speedup_vs_sequential": r["speedup_vs_sequential"],
        "identical_topics": r["identical_topics"],
        "gpu_launches": r["gpu_launches"],
        "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)


def run_heaps(args):
    """The complexity theorem's setting: corpora growing 4x at a time with a
    vocabulary that follows Heaps' law (V = xi N^psi), K fixed.  The theorem
    bounds a sweep's work by sum_i min(K_d, K_v) (the z-step) once the Phi-step,
    whose work grows with K V, is small beside it: reported per token are the
    z-step time and min(K_d, K_v), and the Phi-step's share of the sweep."""
    import torch
    import paper_1704_03581_gb300 as P
    from paper_1704_03581_gb300 import synth

    stream = torch.cuda.Stream()
    rows = []
    for n in [int(x) for x in args.heaps_sizes.split(",")]:
        c = synth.heaps_corpus(n, args.heaps_xi, args.heaps_psi)
        s = P.Sampler(c.w, c.doc_off, K_TOPICS, c.V, ALPHA, BETA, seed=0, stream=stream.cuda_stream)
        s.sweep(args.burnin)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        mins = []
        for e in ev:
            e[0].record(stream)
            P.pulda_phi_step(s.h)
            e[1].record(stream)
            P.pulda_z_step(s.h)
            e[2].record(stream)
            st = s.stats()
            mins.append(st["sum_min"] / max(1, st["tokens"]))
        phi = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
        z = float(np.median([e[1].elapsed_time(e[2]) for e in ev]))
        rows.append({"N": c.N, "V": c.V, "distinct_words": int(np.count_nonzero(np.bincount(c.w, minlength=c.V))),
                     "D": c.D, "z_ns_per_token": 1e6 * z / c.N, "phi_ms": phi, "z_ms": z,
                     "phi_share": phi / (phi + z), "mean_min_kd_kv": float(np.mean(mins)),
                     "nnz_phi": int(st["nnz_phi"]), "sweep_tokens_per_s": c.N / ((phi + z) / 1000.0)})
        s.close()
        print(json.dumps({"progress": f"N={c.N}", "z_ns_per_token": rows[-1]["z_ns_per_token"]}), file=sys.stderr,
              flush=True)
    line = {
        "metric": "sweep cost as the corpus grows with a Heaps'-law vocabulary (complexity theorem)",
        "value": rows[-1]["sweep_tokens_per_s"], "unit": "tokens/s at the largest size", "n_gpus": 1,
        "steps": args.steps, "warmup": args.burnin, "higher_is_better": True, "dtype": "int64",
        "data": "synthetic (LDA generative process, Zipf(1.05) over a V = xi N^psi vocabulary)",
        "config": {"workload": f"N in {args.heaps_sizes}, xi={args.heaps_xi}, psi={args.heaps_psi}",
                   "K": K_TOPICS, "alpha": ALPHA, "beta": BETA, "documents": "lognormal(330, 0.8)"},
        "rows": rows,
    }
    print(json.dumps(line), flush=True)


def serve_continuous(model, reqs, arrivals, sweeps: int, slice_tokens: int, check: int = 10) -> dict:
    """The continuous-batching server fed the requests at their arrival times
    (seconds from the start); latency = arrival to result on the host.  A
    sample of `check` requests is re-run alone (pulda_infer) and must give the
    same topics."""
    import threading
    import paper_1704_03581_gb300 as P
    n = len(arrivals)
    srv = P.Server(model, token_budget=1 << 25, max_slots=8192, slice_tokens=slice_tokens)
    done = {}
    stop = threading.Event()

    def poller():
        deadline = time.monotonic() + 300.0
        while (not stop.is_set() or len(done) < n) and time.monotonic() < deadline:
            for r in srv.poll(max_results=4096, timeout_ms=50):
                done[r["req_id"]] = r
    th = threading.Thread(target=poller)
    th.start()
    t0 = time.monotonic_ns()
    i = 0
    while i < n:
        now = (time.monotonic_ns() - t0) / 1e9
        while i < n and arrivals[i] <= now:
            a, b = int(reqs.doc_off[i]), int(reqs.doc_off[i + 1])
            srv.submit(i, 7919 * i + 1, reqs.w[a:b], sweeps)
            i += 1
        if i < n:
            time.sleep(max(0.0, min(arrivals[i] - now, 0.001)))
    stop.set()
    th.join()
    t_end = max(r["done_ns"] for r in done.values())
    lat = np.array([(done[j]["done_ns"] - t0) / 1e6 - arrivals[j] * 1e3 for j in range(n)])
    toks = int(np.diff(reqs.doc_off)[:n].sum())
    st = srv.stats()
    srv.close()
    same = True
    for j in list(range(0, n, max(1, n // check)))[:check]:
        a, b = int(reqs.doc_off[j]), int(reqs.doc_off[j + 1])
        alone = model.infer(reqs.w[a:b], np.array([0, b - a]), sweeps, seed=7919 * j + 1)
        same &= bool(np.array_equal(alone, done[j]["z"]))
    return {"requests": n, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "docs_per_s": n / ((t_end - t0) / 1e9), "token_sweeps_per_s": toks * sweeps / ((t_end - t0) / 1e9),
            "identical_to_alone": same,
            "server": {"launches": st["launches"], "final_slice": st["slice"],
                       "max_requests_per_launch": st["max_active"],
                       "kernel_share": st["kernel_ns"] / max(1, t_end - t0)}}


def serve_plain(model, reqs, arrivals, sweeps: int, first: int = 0) -> dict:
    """One request at a time through pulda_infer, requests first..first+n-1
    arriving at the given times: latency = arrival to result (queueing
    included); service = the call's own duration."""
    n = len(arrivals)
    t0 = time.monotonic_ns()
    lat, svc = [], []
    for j in range(n):
        now = (time.monotonic_ns() - t0) / 1e9
        if arrivals[j] > now:
            time.sleep(arrivals[j] - now)
        a, b = int(reqs.doc_off[first + j]), int(reqs.doc_off[first + j + 1])
        t1 = time.monotonic_ns()
        model.infer(reqs.w[a:b], np.array([0, b - a]), sweeps, seed=7919 * (first + j) + 1)
        t2 = time.monotonic_ns()
        svc.append((t2 - t1) / 1e6)
        lat.append((t2 - t0) / 1e6 - arrivals[j] * 1e3)
    t_all = (time.monotonic_ns() - t0) / 1e9
    return {"requests": n, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "service_p50_ms": float(np.percentile(svc, 50)), "service_p99_ms": float(np.percentile(svc, 99)),
            "service_mean_ms": float(np.mean(svc)), "docs_per_s": n / t_all}


def plain_capacity(model, reqs, sweeps: int, n: int = 30) -> float:
    """Requests per second that one-at-a-time serving completes back to back
    (the first n requests, no waiting): the highest rate it can sustain."""
    t0 = time.monotonic()
    for j in range(n):
        a, b = int(reqs.doc_off[j]), int(reqs.doc_off[j + 1])
        model.infer(reqs.w[a:b], np.array([0, b - a]), sweeps, seed=7919 * j + 1)
    return n / (time.monotonic() - t0)


def serving_probe(model, V: int, sweeps: int, slice_tokens: int, low_requests: int, high_rate: float,
                  high_seconds: float) -> dict:
    """Both arms on one seeded Poisson trace at half the one-at-a-time arm's
    measured capacity (a rate it sustains), then the continuous arm at a high
    rate: p50/p99 latency, service times, requests served per second."""
    from paper_1704_03581_gb300 import synth
    n_high = int(high_rate * high_seconds)
    reqs, _ = synth.serving_requests(low_requests + n_high + 30, V, rate=1.0)
    cap = plain_capacity(model, reqs, sweeps)
    rate = max(1.0, round(0.5 * cap))
    arrivals = np.cumsum(np.random.default_rng(12).exponential(1.0 / rate, size=low_requests))
    cont_low = serve_continuous(model, reqs, arrivals, sweeps, slice_tokens)
    plain_low = serve_plain(model, reqs, arrivals, sweeps)
    hi_arr = np.cumsum(np.random.default_rng(13).exponential(1.0 / high_rate, size=n_high))
    sub = synth.Corpus(reqs.w[int(reqs.doc_off[low_requests]):],
                       reqs.doc_off[low_requests:] - reqs.doc_off[low_requests], reqs.V, reqs.name)
    cont_high = serve_continuous(model, sub, hi_arr, sweeps, slice_tokens)
    return {"trace": f"Poisson arrivals, lengths lognormal(300, 1.2) clipped to [10, 20000], {sweeps} sweeps per "
                     f"request, the model's Phi after its sweeps",
            "one_at_a_time_capacity_docs_per_s": cap,
            "rate_docs_per_s": rate,
            "continuous": cont_low, "one_at_a_time": plain_low,
            "p99_ratio_plain_over_continuous": plain_low["p99_ms"] / cont_low["p99_ms"],
            "high_rate": dict(cont_high, rate_docs_per_s=high_rate),
            "throughput_ratio_high_over_plain_capacity": cont_high["docs_per_s"] / cap,
            "identical_to_alone": bool(cont_low["identical_to_alone"] and cont_high["identical_to_alone"])}


def run_serving(args):
    """Fold-in requests (lognormal(300, 1.2) tokens clipped to [10, 20000], 50
    sweeps each) arriving as a Poisson process, served against the large
    model's Phi after 50 sweeps: continuous batching at every rate, and one
    request at a time at rates below its measured capacity, on the same
    seeded traces."""
    import paper_1704_03581_gb300 as P
    from paper_1704_03581_gb300 import synth

    corpus = synth.large()
    model = P.Sampler(corpus.w, corpus.doc_off, K_TOPICS, corpus.V, ALPHA, BETA, seed=0,
                      coop_min_len=args.coop_min_len)
    model.sweep(50)
    model.sync()
    rates = [float(r) for r in args.rates.split(",")]
    n_max = int(max(rates) * args.serve_seconds) + args.plain_requests + 30
    reqs, _ = synth.serving_requests(n_max, corpus.V, rate=1.0)
    cap = plain_capacity(model, reqs, args.serve_sweeps)
    plain_rates = [max(1.0, round(f * cap)) for f in (0.25, 0.5, 0.75)]
    results, plains = [], []
    for rate in plain_rates:
        arrivals = np.cumsum(np.random.default_rng(12).exponential(1.0 / rate, size=args.plain_requests))
        c = serve_continuous(model, reqs, arrivals, args.serve_sweeps, args.slice)
        p = serve_plain(model, reqs, arrivals, args.serve_sweeps)
        results.append(dict(c, rate_docs_per_s=rate))
        plains.append(dict(p, rate_docs_per_s=rate))
    for rate in rates:
        n = int(rate * args.serve_seconds)
        arrivals = np.cumsum(np.random.default_rng(11).exponential(1.0 / rate, size=n))
        results.append(dict(serve_continuous(model, reqs, arrivals, args.serve_sweeps, args.slice),
                            rate_docs_per_s=rate))
    model.close()
    low = results[0]
    line = {
        "metric": "serving p50/p99 vs plain (fold-in, 50 sweeps per request, K=1000, V=100000)",
        "value": low["p99_ms"], "unit": "ms (p99 at the lowest rate)", "n_gpus": 1, "steps": len(results),
        "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic requests, lognormal(300, 1.2) tokens clipped to [10, 20000], Poisson arrivals",
        "config": {"workload": "fold-in against the large model's Phi after 50 sweeps", "slice_tokens": args.slice,
                   "coop_min_len": args.coop_min_len, "sweeps_per_request": args.serve_sweeps},
        "one_at_a_time_capacity_docs_per_s": cap,
        "continuous_batching": results,
        "one_at_a_time": plains,
        "p99_ratio_plain_over_continuous": [p["p99_ms"] / c["p99_ms"] for p, c in zip(plains, results)],
        "throughput_ratio_vs_plain_capacity": max(r["docs_per_s"] for r in results) / cap,
    }
    print(json.dumps(line), flush=True)


def main():
    global K_TOPICS
    args = parse()
    K_TOPICS = args.K
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    from paper_1704_03581_gb300 import synth

    if args.impl == "reference":
        if rank != 0:
            return
        corpus = synth.large(D=args.docs)
        run_reference(args, corpus)
        return
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.form in ("batched", "serving", "trace", "sparsity", "heaps"):
        from paper_1704_03581_gb300 import build
        build.build()
        if rank == 0:
            {"batched": run_batched, "serving": run_serving, "trace": run_trace,
             "sparsity": run_sparsity, "heaps": run_heaps}[args.form](args)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1704_03581_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    corpus = synth.large(D=args.docs)
    run_pulda(args, corpus, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
