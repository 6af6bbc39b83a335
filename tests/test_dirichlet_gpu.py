"""Algorithm 1's Dirichlet Phi-step on the GPU, bit-exact with the oracle:
Gamma draws (compared as float bits), row sums (double bits), the kept
entries and their tables, and the z-steps that follow."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1704_03581_gb300 import synth
import paper_1704_03581_gb300 as P
from parity_util import lockstep, oracle_tables_flat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03581_gb300 import build
    build.build()


def random_corpus(seed, D, V, max_len, zipf=1.0):
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, max_len, size=D)
    off = np.zeros(D + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    p = (1.0 + np.arange(V)) ** -zipf
    w = rng.choice(V, size=int(off[-1]), p=p / p.sum()).astype(np.int32)
    return w, off


@pytest.mark.parametrize("path", [0, 1, 2])
def test_tiny_corpus_dirichlet_lockstep(path):
    """K=20 generative corpus, 4 sweeps, every z-step iteration path."""
    c = synth.tiny()
    s, ch = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=5, sweeps=4, path=path, check_counts_every=2,
                     docs_per_warp=1, phi_mode=1)
    s.close()


@pytest.mark.parametrize("K", [1, 33, 1000, 3000])
def test_dirichlet_lockstep_shapes(K):
    """Around the 32-topic words, the 1024 bitmap limit (3000: column path only), rows summed over several chunks."""
    w, off = random_corpus(K, 300, 900, 120)
    alpha = np.random.default_rng(K).uniform(0.05, 1.0, K).astype(np.float32)
    s, ch = lockstep(w, off, K, 900, alpha, 0.02, seed=K, sweeps=2, phi_mode=1)
    s.close()


def test_dirichlet_frequent_word_and_export():
    """A word of more than 2^17 tokens (chunked histogram pass); exported phi equals the oracle's
    and each topic's kept entries carry all but at most V K 2^-24 of its mass."""
    rng = np.random.default_rng(9)
    V, K = 60, 24
    off = np.zeros(301, np.int64)
    np.cumsum(np.full(300, 600), out=off[1:])
    w = np.where(rng.random(int(off[-1])) < 0.8, 0, rng.integers(1, V, int(off[-1]))).astype(np.int32)
    assert (w == 0).sum() > 2 ** 17
    s, ch = lockstep(w, off, K, V, 0.2, 0.05, seed=3, sweeps=2, phi_mode=1)
    col, top, phi = s.phi()
    o = oracle_tables_flat(ch.tables)
    assert np.array_equal(col, o["col_ptr"]) and np.array_equal(top, o["topic"])
    assert np.array_equal(phi.view(np.uint32), o["phi"].view(np.uint32))
    dense = np.zeros((K, V))
    for v in range(V):
        dense[top[col[v]:col[v + 1]], v] = phi[col[v]:col[v + 1]]
    assert np.all(np.abs(dense.sum(axis=1) - 1.0) <= V * K * 2.0 ** -24 + 1e-5)
    s.close()


def test_dirichlet_fold_in_matches_oracle():
    """Fold-in against a Dirichlet Phi: the same z as the oracle's."""
    c = synth.tiny()
    s, ch = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=2, sweeps=2, phi_mode=1)
    w2, off2 = random_corpus(4, 50, c.V, 80)
    z = s.infer(w2, off2, 3, 17)
    zo = O.infer(ch.tables, w2, off2, 3, 17)
    assert np.array_equal(z, zo)
    s.close()


def test_dirichlet_serving():
    """Against a Dirichlet Phi, the server's results equal pulda_infer on each document alone."""
    import time
    c = synth.tiny()
    s = P.Sampler(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=8, phi_mode=1).sweep(2)
    rng = np.random.default_rng(12)
    reqs = [dict(id=i, seed=int(rng.integers(1, 2 ** 62)), words=rng.integers(0, c.V, int(L)).astype(np.int32),
                 sweeps=int(rng.integers(1, 6))) for i, L in enumerate(rng.choice([1, 33, 300, 1000], size=12))]
    srv = P.Server(s, token_budget=4000, max_slots=8, slice_tokens=64)
    for r in reqs:
        srv.submit(r["id"], r["seed"], r["words"], r["sweeps"])
    got, t0 = {}, time.time()
    while len(got) < len(reqs):
        for res in srv.poll(timeout_ms=200):
            assert res["status"] == 0
            got[res["req_id"]] = res["z"]
        assert time.time() - t0 < 120, "server made no progress"
    srv.close()
    for r in reqs:
        alone = s.infer(r["words"], np.array([0, len(r["words"])]), r["sweeps"], seed=r["seed"])
        assert np.array_equal(got[r["id"]], alone)
    s.close()
