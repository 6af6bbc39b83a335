"""Stale-count slices of long documents (an option outside the paper) on the
GPU, bit-exact with the oracle's sliced z-step: every z, the counters, and
the tables the next sweep builds from them."""
import numpy as np
import pytest

from paper_1704_03581_gb300 import synth
import paper_1704_03581_gb300 as P
from parity_util import lockstep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03581_gb300 import build
    build.build()


@pytest.mark.parametrize("slice_len", [1, 37, 100])
def test_tiny_corpus_slices_lockstep(slice_len):
    """Lengths Poisson(100): with 37 or 100 most documents are cut, the last slice ragged; with 1 every token is a slice."""
    c = synth.tiny()
    s, ch = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=4, sweeps=3, check_counts_every=3, slice_len=slice_len)
    s.close()


def test_slices_at_k1000_with_long_documents():
    """K=1000 (dense rows, document side), documents up to 3,000 tokens in slices of 256."""
    rng = np.random.default_rng(17)
    lengths = rng.integers(1, 3000, size=120)
    off = np.zeros(121, np.int64)
    np.cumsum(lengths, out=off[1:])
    V = 5000
    p = (1.0 + np.arange(V)) ** -1.0
    w = rng.choice(V, size=int(off[-1]), p=p / p.sum()).astype(np.int32)
    s, ch = lockstep(w, off, 1000, V, 0.1, 0.01, seed=6, sweeps=2, slice_len=256)
    s.close()


def test_slices_longer_than_every_document_change_nothing():
    """slice_len at least the longest document: the GPU chain equals Algorithm 2's."""
    c = synth.tiny()
    longest = int(np.diff(c.doc_off).max())
    a = P.Sampler(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=9).sweep(3)
    b = P.Sampler(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=9, slice_len=longest).sweep(3)
    assert np.array_equal(a.z(), b.z())
    a.close()
    b.close()
