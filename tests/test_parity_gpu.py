"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1704_03581_gb300 import synth
from parity_util import compare_tables, first_mismatch, lockstep

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


@pytest.mark.parametrize("dpw", [4, 1], ids=["4docs-per-warp", "1doc-per-warp"])
@pytest.mark.parametrize("path", [0, 1, 2])
def test_tiny_corpus_lockstep(path, dpw):
    """K=20, V=1,000, D=1,000, ~100k tokens from the LDA generative process."""
    c = synth.tiny()
    s, ch = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=0, sweeps=6, path=path, check_counts_every=3,
                     docs_per_warp=dpw)
    s.close()


@pytest.mark.parametrize("dpw", [4, 1], ids=["4docs-per-warp", "1doc-per-warp"])
def test_small_corpus_lockstep(dpw):
    """Small-corpus shape: D=1,500, V=12,375, ~1.9M tokens, K=100."""
    c = synth.small()
    s, ch = lockstep(c.w, c.doc_off, 100, c.V, 0.1, 0.01, seed=1, sweeps=3, docs_per_warp=dpw)
    s.close()


@pytest.mark.parametrize("dpw", [4, 1], ids=["4docs-per-warp", "1doc-per-warp"])
@pytest.mark.parametrize("K", [1, 31, 33, 200, 256, 257, 500, 513, 1000, 1024, 1025, 1500, 2048, 2049, 3000])
def test_topic_counts_around_tile_edges(K, dpw):
    """K around the 32-topic words, the 128 topics a lane owns in the grouped
    kernel (1024 its limit), the one-warp kernel's switches from 8 to 16 to 32
    to 64 topics per lane (256 / 512 / 1024), and the 2048 limit of the bitmap
    paths."""
    if dpw == 4 and K > 1024:
        pytest.skip("four documents per warp needs K <= 1024")
    rng = np.random.default_rng(K)
    lengths = rng.integers(0, 90, size=120)
    lengths[3] = 0
    lengths[5] = 1
    lengths[7] = 33
    w, off = corpus_from_lengths(rng, lengths, 700)
    s, _ = lockstep(w, off, K, 700, rng.uniform(0.05, 0.5, K).astype(np.float32), 0.02, seed=K, sweeps=3,
                    check_counts_every=3, docs_per_warp=dpw)
    s.close()


def test_beta_field_chaining_lockstep():
    """beta = 0.001 over K = 3,000 topics and V = 5,000 words: the skip-ahead
    walks of the beta-only entries pass the 1024-entry gap table in about a
    third of their gaps (per word over K, and per dead row over V), so the
    device walk's chaining is compared entry by entry with the oracle's."""
    rng = np.random.default_rng(1001)
    lengths = rng.poisson(40, size=250)
    w, off = corpus_from_lengths(rng, lengths, 5000)
    s, ch = lockstep(w, off, 3000, 5000, 0.1, 0.001, seed=9, sweeps=2, check_counts_every=2)
    assert s.stats()["dead_rows"] > 0
    s.close()


@pytest.mark.parametrize("path", [0, 1, 2])
def test_documents_longer_than_the_grouped_kernel_takes(path):
    """Documents over 65,535 tokens go to the one-document-per-warp kernel in
    the same z-step as the grouped kernel's documents."""
    rng = np.random.default_rng(17)
    lengths = np.concatenate([[70000, 65535, 65536], rng.integers(1, 400, size=37)])
    w, off = corpus_from_lengths(rng, lengths, 500)
    s, _ = lockstep(w, off, 50, 500, 0.1, 0.01, seed=5, sweeps=2, path=path, check_counts_every=2,
                    docs_per_warp=4)
    s.close()


@pytest.mark.parametrize("K", [1, 40])
@pytest.mark.parametrize("longest", [70000, 65535])
def test_count_width_of_the_one_warp_z_step(longest, K):
    """Every document on the one-warp kernel (no cooperative CTAs): with one
    of 70,000 tokens the launch keeps 32-bit counts, with the longest at
    65,535 tokens 16-bit ones -- at K = 1 a count reaches 65,535."""
    rng = np.random.default_rng(longest + K)
    lengths = np.concatenate([[longest, 65535], rng.integers(1, 300, size=30)])
    w, off = corpus_from_lengths(rng, lengths, 400)
    s, _ = lockstep(w, off, K, 400, 0.1, 0.01, seed=6, sweeps=2, check_counts_every=2, coop_min_len=-1)
    s.close()


def test_ragged_and_degenerate_inputs():
    """Empty documents, unused words (empty Phi columns keep their tokens'
    topics), a long document spanning many 32-token batches, and tiny V with
    small beta so whole Phi rows die and are redrawn."""
    rng = np.random.default_rng(5)
    lengths = np.array([0, 1, 2, 0, 31, 32, 33, 1000, 0, 7])
    w, off = corpus_from_lengths(rng, lengths, 3, zipf=0.5)
    s, ch = lockstep(w, off, 12, 6, 0.3, 0.001, seed=9, sweeps=8, check_counts_every=2)
    s.close()


def test_four_documents_per_warp_rejects_large_K():
    import paper_1704_03581_gb300 as P
    with pytest.raises(P.PuldaError):
        P.Sampler(np.zeros(3, np.int32), np.array([0, 3]), 1025, 2, 0.1, 0.01, 0, docs_per_warp=4)


def test_dead_rows_are_redrawn_like_the_oracle():
    rng = np.random.default_rng(6)
    w, off = corpus_from_lengths(rng, np.array([3, 2, 4]), 4)
    total_dead = 0
    s, ch = lockstep(w, off, 9, 4, 0.5, 0.05, seed=3, sweeps=1)
    for it in range(2, 12):
        s.phi_step()
        ch.sweep_index += 1
        ch.phi_step(ch.sweep_index)
        compare_tables(s.word_tables(), ch, f"sweep {it}")
        total_dead += ch.dead_rows
        assert s.stats()["dead_rows"] == ch.dead_rows
        s.z_step()
        ch.z, ch.stats = O.z_step(ch.doc_off, ch.w, ch.z, ch.tables, ch.seed, ch.sweep_index)
        assert not first_mismatch(s.z(), ch.z, off)
    assert total_dead > 20          # the redraw path was exercised
    s.close()


def test_phi_export_and_invariants():
    c = synth.tiny()
    s, ch = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=4, sweeps=2)
    col, top, phi = s.phi()
    o = ch.tables
    mask = np.arange(20)[None, :] < o.ncol[:, None]
    assert np.array_equal(top, o.topic[mask]) and np.array_equal(phi.view(np.uint32), o.phi32[mask].view(np.uint32))
    dense = np.zeros((20, c.V))
    dense[top.astype(np.int64), np.repeat(np.arange(c.V), np.diff(col))] = phi
    assert np.abs(dense.sum(axis=1) - 1).max() < 1e-6
    m = s.m()
    assert np.array_equal(m.sum(axis=1), np.diff(c.doc_off))
    n = s.n()
    assert n.sum() == c.N
    s.close()


def test_resume_from_checkpoint_is_exact():
    c = synth.tiny()
    import paper_1704_03581_gb300 as P
    a = P.Sampler(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=8).sweep(4)
    z4 = a.z()
    a.sweep(3)
    b = P.Sampler(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=8)
    b.set_z(z4, 4)
    b.sweep(3)
    assert np.array_equal(a.z(), b.z())
    a.close(); b.close()


@pytest.mark.parametrize("dpw", [4, 1], ids=["4docs-per-warp", "1doc-per-warp"])
def test_fold_in_matches_oracle(dpw):
    """pulda_infer: Algorithm 2's z-step with Phi held fixed, on new documents."""
    c = synth.tiny()
    s, ch = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=2, sweeps=3, docs_per_warp=dpw)
    new = c.slice_docs(0, 50)
    zg, mg = s.infer(new.w, new.doc_off, 10, seed=77, want_m=True)
    zo = O.infer(ch.tables, new.w, new.doc_off, 10, 77)
    assert not first_mismatch(zg, zo, new.doc_off)
    assert np.array_equal(mg, O.doc_topic(new.doc_off, zo, 20))
    # the chain itself is untouched by a fold-in
    assert np.array_equal(s.z(), ch.z)
    s.close()


def test_large_corpus_sampled_parity():
    """The large workload (D=300,000, V=100,000, ~99M tokens, K=1,000) in the
    launch configuration the benchmark times: one full sweep on the GPU; the
    oracle recomputes the whole Phi-step and the z-step of 3,000 sampled
    documents (documents are independent given Phi), then a fold-in of the
    corpus's longest documents (cooperative z-step) against that Phi."""
    import paper_1704_03581_gb300 as P
    c = synth.large()
    K = 1000
    s = P.Sampler(c.w, c.doc_off, K, c.V, 0.1, 0.01, seed=0)
    z0 = s.z()
    assert np.array_equal(z0, O.init_z(c.N, K, 0))
    s.phi_step()
    ctx = O.Ctx(0.01)
    n = O.count_n(c.w, z0, K, c.V)
    cc, S, dead = O.phi_draw(ctx, n, 0, 1)
    del n
    tab = O.WordTables(cc, S, np.full(K, 0.1, np.float32))

    class _Ch:
        pass
    ch = _Ch()
    ch.K, ch.V, ch.S, ch.c, ch.tables = K, c.V, S, cc, tab
    compare_tables(s.word_tables(), ch, "large sweep 1")
    s.z_step()
    z1 = s.z()
    rng = np.random.default_rng(0)
    docs = np.sort(rng.choice(c.D, size=3000, replace=False))
    for d in docs[:3000]:
        a, b = int(c.doc_off[d]), int(c.doc_off[d + 1])
        zo, _ = O.z_step(np.array([0, b - a], np.int64), c.w[a:b], z0[a:b], tab, 0, 1, index_base=a)
        assert np.array_equal(z1[a:b], zo), f"document {d} differs"
    # fold-in against this Phi at full size: the six longest documents of the
    # corpus go to the cooperative z-step (CTAs), two short ones to one warp each
    L = np.diff(c.doc_off)
    pick = list(np.argsort(-L, kind="stable")[:6]) + [int(docs[0]), int(docs[1])]
    w_new = np.concatenate([c.w[c.doc_off[d]:c.doc_off[d + 1]] for d in pick])
    off_new = np.zeros(len(pick) + 1, np.int64)
    np.cumsum(L[pick], out=off_new[1:])
    zg = s.infer(w_new, off_new, 2, seed=13)
    zo = O.infer(tab, w_new, off_new, 2, 13)
    assert not first_mismatch(zg, zo, off_new)
    s.close()


def test_large_corpus_steady_state_parity():
    """The large workload in the benchmark's launch configuration after 30
    sweeps on the GPU (the benchmark times sweeps 31-50): Phi is sparser than
    after the uniform start, the document/column sides and the dense rows fall
    as in the timed window.  From the GPU's topics after sweep 30 the oracle,
    on all host cores, recomputes sweep 31 in full: every Poisson count, row
    sum and table, then the z-step of every document -- all 99M topics and the
    six z-step counters compared exactly (the 100 longest documents and the
    cooperative ones among them)."""
    import paper_1704_03581_gb300 as P
    c = synth.large()
    K = 1000
    T = O.host_threads()
    s = P.Sampler(c.w, c.doc_off, K, c.V, 0.1, 0.01, seed=0)
    s.sweep(30)
    z30 = s.z()
    assert s.stats()["sweep"] == 30
    s.phi_step()
    ctx = O.Ctx(0.01)
    n = O.count_n(c.w, z30, K, c.V, threads=T)
    cc, S, dead = O.phi_draw(ctx, n, 0, 31, threads=T)
    del n
    tab = O.WordTables(cc, S, np.full(K, 0.1, np.float32), threads=T)

    class _Ch:
        pass
    ch = _Ch()
    ch.K, ch.V, ch.S, ch.c, ch.tables = K, c.V, S, cc, tab
    compare_tables(s.word_tables(), ch, "large sweep 31")
    assert s.stats()["dead_rows"] == dead
    s.z_step()
    z31, st = s.z(), s.stats()
    zo, sto = O.z_step(c.doc_off, c.w, z30, tab, 0, 31, threads=T)
    L = np.diff(c.doc_off)
    longest = np.argsort(-L, kind="stable")[:100]
    for d in longest:
        a, b = int(c.doc_off[d]), int(c.doc_off[d + 1])
        assert np.array_equal(z31[a:b], zo[a:b]), f"long document {d} ({b - a} tokens) differs"
    assert not first_mismatch(z31, zo, c.doc_off)
    assert [st["tokens"], st["a_branch"], st["sum_min"], st["zero_mass"], st["sum_inter"], st["docside"]] == \
        [int(x) for x in sto]
    s.close()


@pytest.mark.parametrize("K,phi_mode", [(20, 0), (1000, 0), (33, 1)])
def test_sort_count_path_lockstep(K, phi_mode):
    """count_path 1: n rebuilt by radix-sorting the tokens' (word, topic)
    keys instead of per-word histograms; every count, draw, table and topic
    as the oracle's (empty documents and unused words included; keys of 15,
    20 and 15 bits: two or three 8-bit digit passes)."""
    rng = np.random.default_rng(70 + K)
    lengths = rng.integers(0, 300, size=150)
    lengths[[2, 4]] = [0, 1]
    w, off = corpus_from_lengths(rng, lengths, 900)
    s, _ = lockstep(w, off, K, 900, 0.1, 0.01, seed=K, sweeps=3, check_counts_every=3, phi_mode=phi_mode,
                    count_path=1)
    s.close()


@pytest.mark.parametrize("K,dpw,phi_mode,coop", [(20, 1, 0, 0), (1000, 1, 0, 150), (3000, 1, 0, 0), (200, 4, 0, 0),
                                                 (33, 1, 1, 0)])
def test_packed_alias_slots_lockstep(K, dpw, phi_mode, coop):
    """alias_layout 2: the z-step takes each alias draw from one packed
    8-byte slot {threshold, topic | alias topic << 16} that the table pass
    writes beside the threshold and topic arrays.  Every table, draw, count
    and topic as the oracle's: the one-warp kernel at 8 and 32 topics per lane
    and past the bitmap limit, the cooperative kernel on documents of at least
    150 tokens, four documents per warp, the Dirichlet Phi; then a fold-in."""
    rng = np.random.default_rng(90 + K)
    lengths = rng.integers(0, 300, size=150)
    lengths[[2, 4]] = [0, 1]
    w, off = corpus_from_lengths(rng, lengths, 900)
    s, ch = lockstep(w, off, K, 900, 0.1, 0.01, seed=K, sweeps=3, check_counts_every=3, phi_mode=phi_mode,
                     docs_per_warp=dpw, coop_min_len=coop, alias_layout=2)
    new_off = off[:21] - off[0]
    new_w = w[:new_off[-1]]
    zg = s.infer(new_w, new_off, 5, seed=5)
    zo = O.infer(ch.tables, new_w, new_off, 5, 5)
    assert not first_mismatch(zg, zo, new_off)
    s.close()


def test_sort_count_path_small_corpus():
    """The small corpus (1.9M tokens, K=100): words with up to ~10^5 tokens,
    the sort's multi-block scans over every tile."""
    c = synth.small()
    s, _ = lockstep(c.w, c.doc_off, 100, c.V, 0.1, 0.01, seed=1, sweeps=2, count_path=1)
    s.close()


def test_z_layout_follows_the_measured_rule():
    """Auto takes one document per warp at every K; 4 forces four
    (K <= 1024), the column-only path one; the longest documents go to CTAs
    either way."""
    import paper_1704_03581_gb300 as P
    rng = np.random.default_rng(5)
    lengths = np.concatenate([[4000], rng.integers(1, 200, size=200)])
    w, off = corpus_from_lengths(rng, lengths, 800)
    for K, kw, dpw in [(20, {}, 1), (256, {}, 1), (257, {}, 1), (1000, {}, 1), (1000, dict(docs_per_warp=4), 4),
                       (20, dict(docs_per_warp=4), 4), (100, dict(docs_per_warp=1), 1), (100, dict(zstep_path=1), 1)]:
        s = P.Sampler(w, off, K, 800, 0.1, 0.01, seed=1, **kw)
        lay = s.z_layout()
        assert lay["docs_per_warp"] == dpw, (K, kw, lay)
        assert lay["coop_docs"] == 1, (K, kw, lay)          # the 4,000-token document is above max(256, N / div)
        s.close()
