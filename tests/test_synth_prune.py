"""Vocabulary pruning of the synthetic corpora (rare-word threshold, top
TF-IDF words), checked against per-document loops."""
import math

import numpy as np

from paper_1704_03581_gb300 import synth


def _corpus_with_empty_docs():
    rng = np.random.default_rng(11)
    lengths = rng.integers(0, 30, size=60)
    lengths[[0, 7, 59]] = 0
    off = np.zeros(61, np.int64)
    np.cumsum(lengths, out=off[1:])
    w = (rng.zipf(1.6, size=int(off[-1])) % 40).astype(np.int32)
    return synth.Corpus(w, off, 40, "t")


def _docs(c):
    return [c.w[c.doc_off[d]:c.doc_off[d + 1]].tolist() for d in range(c.D)]


def test_keep_words_matches_per_document_filter():
    c = _corpus_with_empty_docs()
    keep = np.arange(c.V) % 3 != 1
    p = synth.keep_words(c, keep, "p")
    ids = {v: i for i, v in enumerate(np.flatnonzero(keep))}
    want = [[ids[v] for v in doc if keep[v]] for doc in _docs(c)]
    assert p.D == c.D and p.V == int(keep.sum())
    assert _docs(p) == want


def test_rare_word_threshold():
    c = _corpus_with_empty_docs()
    cnt = {v: 0 for v in range(c.V)}
    for v in c.w.tolist():
        cnt[v] += 1
    for t in (1, 2, 5, 20):
        p = synth.rare_word_pruned(c, t)
        assert p.V == sum(1 for v in cnt if cnt[v] >= t)
        assert p.N == sum(n for n in cnt.values() if n >= t)
        assert np.all(np.bincount(p.w, minlength=p.V) >= t) or p.N == 0


def test_tfidf_and_top_words():
    c = _corpus_with_empty_docs()
    docs = _docs(c)
    w0 = c.w.copy()
    s = synth.tfidf(c)
    assert np.array_equal(c.w, w0)                       # the corpus is left as it was
    for v in range(c.V):
        n = sum(doc.count(v) for doc in docs)
        df = sum(1 for doc in docs if v in doc)
        assert math.isclose(s[v], n * math.log(c.D / df) if df else 0.0, rel_tol=1e-12, abs_tol=0.0)
    p = synth.tfidf_pruned(c, 10)
    kept = sorted(range(c.V), key=lambda v: (-s[v], v))[:10]
    ids = {v: i for i, v in enumerate(sorted(kept))}
    assert p.V == 10 and _docs(p) == [[ids[v] for v in doc if v in ids] for doc in docs]


def test_heaps_corpus_follows_the_law():
    """V = xi N^psi words (the complexity theorem's assumption), about the
    target number of tokens, and no word id outside the vocabulary."""
    from paper_1704_03581_gb300 import synth
    assert synth.heaps_vocabulary(10 ** 6, 20.0, 0.5) == 20000
    assert synth.heaps_vocabulary(4 * 10 ** 6, 20.0, 0.5) == 40000
    c = synth.heaps_corpus(250_000, 20.0, 0.5, K=50)
    assert c.V == synth.heaps_vocabulary(250_000, 20.0, 0.5) == 10000
    assert abs(c.N - 250_000) / 250_000 < 0.1
    assert c.w.min() >= 0 and c.w.max() < c.V
    d = synth.heaps_corpus(1_000_000, 20.0, 0.5, K=50)
    assert d.V == 2 * c.V                     # 4x the tokens, 2x the words at psi = 1/2
