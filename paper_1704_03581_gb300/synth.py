"""Seeded synthetic corpora drawn from the LDA generative process.

The paper's corpora (Enron, NYT, PubMed; Table "corpora" in Section 4) are not
available here, so every workload is synthetic and drawn from the LDA model
itself (Figure "lda-dag"): theta_d ~ Dir(alpha_gen), phi_k ~ Dir(b * F),
z ~ Cat(theta_d), w ~ Cat(phi_z).  F is either uniform (the tiny corpus) or a
Zipf(s) law over a seeded permutation of the word ids, with concentration
b = 0.05 V, so frequent words appear in every topic and rare words in few --
the sparsity structure the doubly sparse sampler exploits.

This module holds no part of the sampler's arithmetic: it only produces the
inputs (word ids in document order and document offsets) that both the CUDA
path and the CPU oracle consume.
"""
from __future__ import annotations

import dataclasses
import math
import os
import tempfile

import numpy as np


@dataclasses.dataclass
class Corpus:
    """A corpus in CSR form: ``w[doc_off[d]:doc_off[d+1]]`` are document d's
    word ids, in position order."""

    w: np.ndarray        # int32 [N]
    doc_off: np.ndarray  # int64 [D+1]
    V: int
    name: str = ""

    @property
    def D(self) -> int:
        return int(self.doc_off.shape[0] - 1)

    @property
    def N(self) -> int:
        return int(self.w.shape[0])

    def slice_docs(self, d0: int, d1: int) -> "Corpus":
        a, b = int(self.doc_off[d0]), int(self.doc_off[d1])
        return Corpus(self.w[a:b].copy(), (self.doc_off[d0:d1 + 1] - a).astype(np.int64), self.V,
                      f"{self.name}[{d0}:{d1}]")


def lognormal_lengths(rng: np.random.Generator, D: int, mean: float, log_sd: float,
                      lo: int = 1, hi: int | None = None) -> np.ndarray:
    """Document lengths with arithmetic mean ``mean`` and log-sd ``log_sd``:
    mu = ln(mean) - log_sd^2 / 2, rounded, floored at ``lo``, capped at ``hi``."""
    mu = math.log(mean) - 0.5 * log_sd * log_sd
    x = np.rint(rng.lognormal(mu, log_sd, size=D)).astype(np.int64)
    x = np.maximum(x, lo)
    if hi is not None:
        x = np.minimum(x, hi)
    return x


def zipf_base(rng: np.random.Generator, V: int, s: float) -> np.ndarray:
    """Zipf(s) probabilities over a seeded permutation of 0..V-1."""
    ranks = rng.permutation(V)
    p = (1.0 + ranks.astype(np.float64)) ** (-s)
    return p / p.sum()


def _dirichlet_rows(rng: np.random.Generator, shape_row: np.ndarray, rows: int) -> np.ndarray:
    g = rng.standard_gamma(np.broadcast_to(shape_row, (rows, shape_row.shape[0])))
    tot = g.sum(axis=1, keepdims=True)
    tot[tot <= 0] = 1.0
    g /= tot
    return g


def lda_corpus(seed: int, K: int, V: int, lengths: np.ndarray, alpha_gen: float,
               phi_shape: np.ndarray, name: str = "", doc_chunk: int = 8192,
               phi_seed: int | None = None) -> Corpus:
    """Draw a corpus from the LDA generative process.

    ``phi_shape`` is the Dirichlet parameter vector (length V) shared by every
    topic's word distribution; ``alpha_gen`` the symmetric document-topic
    parameter; ``lengths`` the document lengths.  The topics are drawn from
    ``phi_seed`` (default ``seed + 1``), the rest from ``seed``, so two corpora
    can share topics.
    """
    rng = np.random.default_rng(seed)
    phi_rng = np.random.default_rng(seed + 1 if phi_seed is None else phi_seed)
    lengths = np.asarray(lengths, dtype=np.int64)
    D = lengths.shape[0]
    doc_off = np.zeros(D + 1, dtype=np.int64)
    np.cumsum(lengths, out=doc_off[1:])
    N = int(doc_off[-1])
    phi = _dirichlet_rows(phi_rng, np.asarray(phi_shape, dtype=np.float64), K)
    z = np.empty(N, dtype=np.int32)
    alpha_row = np.full(K, alpha_gen, dtype=np.float64)
    for d0 in range(0, D, doc_chunk):
        d1 = min(D, d0 + doc_chunk)
        nd = d1 - d0
        theta = _dirichlet_rows(rng, alpha_row, nd)
        cum = np.cumsum(theta, axis=1)
        cum[:, -1] = 1.0
        flat = (cum + np.arange(nd, dtype=np.float64)[:, None]).ravel()
        a, b = int(doc_off[d0]), int(doc_off[d1])
        tok_doc = np.repeat(np.arange(nd, dtype=np.int64), lengths[d0:d1])
        u = rng.random(b - a) + tok_doc
        k = np.searchsorted(flat, u, side="right") - tok_doc * K
        z[a:b] = np.clip(k, 0, K - 1)
    w = np.empty(N, dtype=np.int32)
    order = np.argsort(z, kind="stable")
    counts = np.bincount(z, minlength=K)
    start = 0
    for k in range(K):
        c = int(counts[k])
        if c:
            w[order[start:start + c]] = rng.choice(V, size=c, p=phi[k])
        start += c
    return Corpus(w, doc_off, V, name)


# --------------------------------------------------------------------------
# The workloads.  Sizes follow the five configurations the sampler is
# measured on; seeds are fixed so every run sees the same corpus.
# --------------------------------------------------------------------------

ALPHA = 0.1
BETA = 0.01


def tiny(seed: int = 1) -> Corpus:
    """K=20, V=1,000, D=1,000, lengths Poisson(100), phi_k ~ Dir(0.01),
    theta_d ~ Dir(0.1): the full generative process (~100k tokens)."""
    rng = np.random.default_rng(seed)
    lengths = rng.poisson(100, size=1000)
    return lda_corpus(seed + 1000, 20, 1000, lengths, 0.1, np.full(1000, 0.01), "tiny K=20 V=1000 D=1000")


def zipf_corpus(seed: int, K: int, V: int, D: int, mean_len: float, log_sd: float, s: float,
                name: str, hi: int | None = None) -> Corpus:
    rng = np.random.default_rng(seed)
    lengths = lognormal_lengths(rng, D, mean_len, log_sd, 1, hi)
    F = zipf_base(np.random.default_rng(seed + 7), V, s)
    return lda_corpus(seed + 1000, K, V, lengths, 0.1, 0.05 * V * F, name, phi_seed=seed + 11)


def small(seed: int = 2) -> Corpus:
    """D=1,500, V=12,375, lengths lognormal(mean 1,290, log-sd 0.5), Zipf(1.0),
    generated with K=100 topics (~1.9M tokens)."""
    return zipf_corpus(seed, 100, 12375, 1500, 1290.0, 0.5, 1.0, "small D=1500 V=12375 K=100")


GENERATOR_VERSION = 1


def _cached(key: str, make) -> Corpus:
    """Drawing the large corpus takes about a minute; keep one copy per
    machine (``PULDA_SYNTH_CACHE``, default /tmp/pulda_synth_cache)."""
    d = os.environ.get("PULDA_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "pulda_synth_cache"))
    path = os.path.join(d, f"{key}_v{GENERATOR_VERSION}.npz")
    if os.path.exists(path):
        try:
            with np.load(path) as f:
                return Corpus(f["w"], f["doc_off"], int(f["V"]), str(f["name"]))
        except Exception:
            pass
    c = make()
    try:
        os.makedirs(d, exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp.npz"
        np.savez(tmp, w=c.w, doc_off=c.doc_off, V=c.V, name=c.name)
        os.replace(tmp, path)
    except OSError:
        pass
    return c


def large(seed: int = 3, D: int = 300_000) -> Corpus:
    """D=300,000, V=100,000, lengths lognormal(mean 330, log-sd 0.8),
    Zipf(1.05), generated with K=1,000 topics (~99M tokens)."""
    return _cached(f"large_s{seed}_D{D}", lambda: zipf_corpus(seed, 1000, 100_000, D, 330.0, 0.8, 1.05,
                                                              f"large D={D} V=100000 K=1000"))


def heaps_vocabulary(N: int, xi: float = 20.0, psi: float = 0.5) -> int:
    """Heaps' law, the assumption of the paper's complexity theorem: a corpus
    of N tokens has V = xi N^psi distinct words (for most languages
    5 < xi < 50 and 0.4 < psi < 0.6)."""
    return max(1, int(round(xi * float(N) ** psi)))


def heaps_corpus(N_target: int, xi: float = 20.0, psi: float = 0.5, K: int = 1000, mean_len: float = 330.0,
                 log_sd: float = 0.8, s: float = 1.05, seed: int = 6) -> Corpus:
    """A corpus of about N_target tokens whose vocabulary follows Heaps' law:
    V = heaps_vocabulary(N_target, xi, psi) words with Zipf(s) frequencies,
    documents lognormal(mean_len, log_sd), drawn from the LDA generative
    process with K topics (the large corpus's recipe at another size)."""
    D = max(1, int(round(N_target / mean_len)))
    V = heaps_vocabulary(N_target, xi, psi)
    return zipf_corpus(seed, K, V, D, mean_len, log_sd, s, f"heaps N~{N_target} V={V} xi={xi} psi={psi}")


def batched_specs(n_chains: int = 32, seed: int = 4) -> list[dict]:
    """Shapes of the batched-chains workload: D log-uniform in [1e3, 1e5],
    mean length log-uniform in [50, 2000], V log-uniform in [5e3, 5e4],
    K uniform over {50, 100, 200, 500}; chain seeds 100.."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_chains):
        out.append(dict(
            D=int(round(math.exp(rng.uniform(math.log(1e3), math.log(1e5))))),
            mean_len=float(math.exp(rng.uniform(math.log(50), math.log(2000)))),
            V=int(round(math.exp(rng.uniform(math.log(5e3), math.log(5e4))))),
            K=int(rng.choice([50, 100, 200, 500])),
            seed=100 + c,
        ))
    return out


def batched_corpus(spec: dict, scale: float = 1.0) -> Corpus:
    D = max(1, int(round(spec["D"] * scale)))
    key = f"chain_s{spec['seed']}_D{D}_V{spec['V']}_K{spec['K']}_L{spec['mean_len']:.6g}"
    return _cached(key, lambda: zipf_corpus(spec["seed"], spec["K"], spec["V"], D, spec["mean_len"], 0.8, 1.0,
                                            f"chain{spec['seed']} D={D} V={spec['V']} K={spec['K']}"))


def _batched_one(args) -> int:
    spec, scale = args
    return batched_corpus(spec, scale).N


def batched_corpora(specs: list[dict], scale: float = 1.0, workers: int = 0) -> list[Corpus]:
    """Every chain's corpus, drawn by ``workers`` processes at once (0 = the
    host's cores, at most one per chain) into the on-disk cache, then loaded.
    The pool uses the spawn start method, so it is safe after CUDA has started
    in this process."""
    import multiprocessing as mp
    if workers == 0:
        try:
            workers = len(os.sched_getaffinity(0))
        except AttributeError:
            workers = os.cpu_count() or 1
    workers = max(1, min(workers, len(specs)))
    if workers > 1:
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_batched_one, [(sp, scale) for sp in sorted(specs, key=lambda x: -x["D"] * x["mean_len"])])
    return [batched_corpus(sp, scale) for sp in specs]


def serving_requests(n: int, V: int, seed: int = 5, mean_len: float = 300.0, log_sd: float = 1.2,
                     lo: int = 10, hi: int = 20000, rate: float = 5000.0, K_gen: int = 1000) -> tuple[Corpus, np.ndarray]:
    """Fold-in requests: lengths lognormal(mean 300, log-sd 1.2) clipped to
    [10, 20000], words from the large corpus's generator shape, Poisson
    arrivals at ``rate`` docs/s.  Returns the requests as a corpus (one
    document per request) and the arrival times in seconds."""
    rng = np.random.default_rng(seed)
    lengths = lognormal_lengths(rng, n, mean_len, log_sd, lo, hi)
    F = zipf_base(np.random.default_rng(3 + 7), V, 1.05)       # the large corpus's word law
    corpus = lda_corpus(seed + 1000, K_gen, V, lengths, 0.1, 0.05 * V * F, f"requests n={n}",
                        phi_seed=3 + 11)                          # and its topics
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    return corpus, arrivals


# ------------------------------------------------------------------ vocabulary pruning
# The paper's runtime study over rare-word thresholds, vocabulary sizes and data
# sizes (Section 5, the figure on sparsity) prunes a corpus before sampling:
# words seen fewer than a threshold number of times are removed, or only the
# words with the highest TF-IDF values are kept.  These helpers apply the same
# pruning to a synthetic corpus.

def keep_words(c: Corpus, keep: np.ndarray, name: str) -> Corpus:
    """The corpus restricted to the words with ``keep[v]`` true, renumbered
    0..V'-1 in ascending original id.  Tokens of dropped words are removed
    from their documents (positions close up); every document is kept, so a
    document may become empty."""
    keep = np.asarray(keep, dtype=bool)
    assert keep.shape == (c.V,)
    new_id = np.cumsum(keep, dtype=np.int64) - 1
    mask = keep[c.w]
    kept_before = np.zeros(c.N + 1, np.int64)          # kept tokens before each position
    np.cumsum(mask, out=kept_before[1:])
    off = kept_before[c.doc_off]
    return Corpus(new_id[c.w[mask]].astype(np.int32), off, int(keep.sum()), name)


def word_counts(c: Corpus) -> np.ndarray:
    return np.bincount(c.w, minlength=c.V).astype(np.int64)


def document_frequency(c: Corpus) -> np.ndarray:
    """df[v] = number of documents that contain word v at least once."""
    import scipy.sparse
    m = scipy.sparse.csr_matrix((np.ones(c.N, np.int32), c.w, c.doc_off), shape=(c.D, c.V), copy=True)
    m.sum_duplicates()           # one entry per (document, word) pair; sorts the copy, not c.w
    return np.bincount(m.indices, minlength=c.V).astype(np.int64)


def tfidf(c: Corpus) -> np.ndarray:
    """Corpus-level TF-IDF of each word: its count times ln(D / df), 0 for a
    word that does not occur."""
    n, df = word_counts(c), document_frequency(c)
    out = np.zeros(c.V, np.float64)
    seen = df > 0
    out[seen] = n[seen] * np.log(c.D / df[seen])
    return out


def rare_word_pruned(c: Corpus, threshold: int) -> Corpus:
    """Words that occur fewer than ``threshold`` times removed."""
    return keep_words(c, word_counts(c) >= threshold, f"{c.name} rare<{threshold} removed")


def tfidf_pruned(c: Corpus, V_keep: int, scores: np.ndarray | None = None) -> Corpus:
    """The ``V_keep`` words of highest TF-IDF kept (ties: the smaller id)."""
    s = tfidf(c) if scores is None else scores
    order = np.lexsort((np.arange(c.V), -s))
    keep = np.zeros(c.V, bool)
    keep[order[:min(V_keep, c.V)]] = True
    return keep_words(c, keep, f"{c.name} top-{V_keep} TF-IDF")
