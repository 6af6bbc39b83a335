"""The log-posterior diagnostic (Section 5) on the GPU against the oracle.

Both sides sum the same lgamma terms in double, in different orders and with
different lgamma implementations, so they agree to the worst-case bound of
recursive summation: |error| <= (n + c) * eps * sum |term| per side, n the
number of terms and c a few ulps for each lgamma.  The tests compute
sum |term| from the counts and allow twice that bound.
"""
import numpy as np
import pytest
from scipy.special import gammaln

from oracle import oracle as O
from paper_1704_03581_gb300 import synth
import paper_1704_03581_gb300 as P

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03581_gb300 import build
    build.build()


def bound(doc_off, w, z, K, V, alpha, beta):
    """Twice the worst-case summation error of either side."""
    a = np.broadcast_to(np.asarray(alpha, np.float32), (K,)).astype(np.float64)
    D = doc_off.shape[0] - 1
    d_of = np.repeat(np.arange(D, dtype=np.int64), np.diff(doc_off))
    zz = z.astype(np.int64)
    dk, m = np.unique(d_of * K + zz, return_counts=True)
    kv, n = np.unique(zz * V + w.astype(np.int64), return_counts=True)
    ak = a[dk % K]
    terms = np.abs(gammaln(ak + m) - gammaln(ak)).sum() + np.abs(gammaln(beta + n) - gammaln(beta)).sum()
    A, lens = a.sum(), np.diff(doc_off).astype(np.float64)
    nk = np.bincount(zz, minlength=K).astype(np.float64)
    terms += np.abs(gammaln(A) - gammaln(A + lens)).sum() + np.abs(gammaln(V * beta) - gammaln(V * beta + nk)).sum()
    n_terms = m.size + n.size + D + K
    return 2.0 * (n_terms + 16) * EPS * (terms + 1.0)


def check(s, doc_off, w, K, V, alpha, beta):
    got = s.log_posterior()
    z = s.z()
    want = O.log_posterior(doc_off, w, z, K, V, alpha, float(np.float32(beta)))
    tol = bound(doc_off, w, z, K, V, alpha, float(np.float32(beta)))
    assert np.all(np.abs(got - want) <= tol), (got, want, tol)
    again = s.log_posterior()
    assert np.array_equal(got.view(np.uint64), again.view(np.uint64)), "not reproducible"
    return got


def test_tiny_corpus_log_posterior_over_sweeps():
    """K=20 generative corpus: initial topics and after 2, 5 sweeps; the trace rises from the uniform start."""
    c = synth.tiny()
    s = P.Sampler(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=3)
    lp0 = check(s, c.doc_off, c.w, 20, c.V, 0.1, 0.01)
    s.sweep(2)
    check(s, c.doc_off, c.w, 20, c.V, 0.1, 0.01)
    s.sweep(3)
    lp5 = check(s, c.doc_off, c.w, 20, c.V, 0.1, 0.01)
    assert lp5[0] > lp0[0]
    s.close()


@pytest.mark.parametrize("K", [1, 31, 1000, 3000, 16384])
def test_log_posterior_shapes(K):
    """Every shared-memory layout of the per-document kernel (K up to 16,384), empty documents, asymmetric alpha."""
    rng = np.random.default_rng(K)
    lengths = rng.integers(0, 300, size=400)
    lengths[::37] = 0
    off = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    V = 2000
    w = rng.integers(0, V, int(off[-1])).astype(np.int32)
    alpha = rng.uniform(0.05, 2.0, K).astype(np.float32)
    s = P.Sampler(w, off, K, V, alpha, 0.02, seed=7)
    check(s, off, w, K, V, alpha, 0.02)
    s.sweep(2)
    check(s, off, w, K, V, alpha, 0.02)
    s.close()


def test_log_posterior_with_a_frequent_word():
    """A word with more than 2^17 tokens takes the chunked histogram pass."""
    rng = np.random.default_rng(5)
    V, K = 50, 40
    lengths = np.full(300, 600)
    off = np.zeros(301, np.int64)
    np.cumsum(lengths, out=off[1:])
    w = np.where(rng.random(int(off[-1])) < 0.8, 0, rng.integers(1, V, int(off[-1]))).astype(np.int32)
    assert (w == 0).sum() > 2 ** 17
    s = P.Sampler(w, off, K, V, 0.1, 0.05, seed=2)
    s.sweep(1)
    check(s, off, w, K, V, 0.1, 0.05)
    s.close()
