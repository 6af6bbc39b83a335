"""The cooperative z-step (one CTA of four warps per long document, token by
token) against the oracle: the same topics, counts and counters as Algorithm 2
resampling each document in order."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1704_03581_gb300 import synth
from parity_util import first_mismatch, lockstep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03581_gb300 import build
    build.build()


def corpus_from_lengths(rng, lengths, V, zipf=1.0):
    off = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    p = (1.0 + np.arange(V)) ** -zipf
    w = rng.choice(V, size=int(off[-1]), p=p / p.sum()).astype(np.int32)
    return w, off


@pytest.mark.parametrize("path", [0, 1, 2])
def test_tiny_corpus_every_document_cooperative(path):
    """K=20: one bitmap word, so only the first 32 of the CTA's 128 slots own topics."""
    c = synth.tiny()
    s, _ = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=3, sweeps=4, path=path, check_counts_every=2,
                    coop_min_len=1)
    s.close()


@pytest.mark.parametrize("K", [1, 31, 33, 129, 200, 513, 1000, 1024, 1025, 3000, 16384])
def test_topic_counts_around_slot_edges(K):
    """K around the 32-topic words, the 128 slots (R = 1, 2, 4, 8 topics per slot),
    the 1024 limit of the document side and the largest K (m_d beyond 48 KB of
    shared memory); empty, one-token and 32/33-token documents beside long ones."""
    rng = np.random.default_rng(100 + K)
    lengths = rng.integers(0, 700, size=40)
    lengths[[3, 5, 7, 9]] = [0, 1, 32, 33]
    lengths[0] = 3000
    w, off = corpus_from_lengths(rng, lengths, 900)
    s, _ = lockstep(w, off, K, 900, rng.uniform(0.05, 0.5, K).astype(np.float32), 0.02, seed=K, sweeps=3,
                    check_counts_every=3, coop_min_len=1)
    s.close()


def test_long_and_short_documents_in_the_same_pass():
    """Documents of at least 300 tokens on CTAs while the rest run one per warp
    on the second stream, joined before the counters are read."""
    rng = np.random.default_rng(31)
    lengths = np.concatenate([rng.integers(300, 4000, size=12), rng.integers(0, 300, size=300)])
    rng.shuffle(lengths)
    w, off = corpus_from_lengths(rng, lengths, 2000)
    for path in (0, 1, 2):
        s, _ = lockstep(w, off, 300, 2000, 0.1, 0.01, seed=path, sweeps=2, path=path, check_counts_every=2,
                        coop_min_len=300)
        s.close()


def test_small_corpus_automatic_threshold():
    """Small-corpus shape (D=1,500, ~1.9M tokens, K=100): the automatic threshold
    (N / 8000 = 236, at least 256 tokens) sends most documents to the cooperative kernel."""
    c = synth.small()
    assert (np.diff(c.doc_off) >= max(256, c.N // 8000 + 1)).mean() > 0.9
    s, _ = lockstep(c.w, c.doc_off, 100, c.V, 0.1, 0.01, seed=2, sweeps=2, coop_min_len=0)
    s.close()


def test_fold_in_cooperative():
    c = synth.tiny()
    s, ch = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=2, sweeps=2, coop_min_len=50)
    new = c.slice_docs(0, 60)
    zg = s.infer(new.w, new.doc_off, 8, seed=71)
    zo = O.infer(ch.tables, new.w, new.doc_off, 8, 71)
    assert not first_mismatch(zg, zo, new.doc_off)
    s.close()


def test_cooperative_and_one_warp_give_the_same_chain():
    """The large model's K=1,000 on 2,000 of its documents (the longest over
    7,000 tokens): ten sweeps with every document on one warp, and with every
    document over 64 tokens on a CTA."""
    import paper_1704_03581_gb300 as P
    base = synth.large()
    L = np.diff(base.doc_off)
    pick = np.sort(np.concatenate([np.argsort(-L, kind="stable")[:20], np.arange(1980)]))
    pick = np.unique(pick)
    w = np.concatenate([base.w[base.doc_off[d]:base.doc_off[d + 1]] for d in pick])
    off = np.zeros(len(pick) + 1, np.int64)
    np.cumsum(L[pick], out=off[1:])
    zs = []
    for coop in (-1, 64):
        s = P.Sampler(w, off, 1000, base.V, 0.1, 0.01, seed=5, coop_min_len=coop)
        s.sweep(10)
        zs.append((s.z(), s.stats()))
        s.close()
    assert not first_mismatch(zs[0][0], zs[1][0], off)
    for k in ("tokens", "a_branch", "sum_min", "zero_mass", "sum_inter", "docside", "nnz_phi"):
        assert zs[0][1][k] == zs[1][1][k], k
