"""Batched chains: every chain of a batch equals, bit for bit, the chain a
single handle with the same arguments runs (and hence the oracle), whatever
the z-step CTA size the autotuner picks and across CUDA-graph replays."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03581_gb300 import build
    build.build()


def make_chains():
    """Uneven chains: K from 1 to 1500 (bitmap and column paths, the largest K
    sizing shared memory), V, D, lengths, alpha, beta and seeds all differ."""
    rng = np.random.default_rng(3)
    out = []
    for i, (K, V, D, mean) in enumerate([(1, 50, 10, 5), (37, 400, 300, 40), (100, 2000, 120, 300),
                                         (500, 3000, 60, 150), (1024, 800, 40, 90), (1500, 1200, 80, 60)]):
        lengths = rng.poisson(mean, size=D)
        lengths[0] = 0
        off = np.zeros(D + 1, np.int64)
        np.cumsum(lengths, out=off[1:])
        p = (1.0 + np.arange(V)) ** -1.0
        w = rng.choice(V, size=int(off[-1]), p=p / p.sum()).astype(np.int32)
        alpha = rng.uniform(0.05, 0.5, K).astype(np.float32)
        out.append(dict(w=w, doc_off=off, K=K, V=V, alpha=alpha, beta=float(rng.uniform(0.005, 0.05)), seed=100 + i))
    return out


@pytest.mark.parametrize("warps,coop,form", [(0, 0, 0), (0, -1, 0), (4, -1, 0), (4, 64, 0), (2, 1, 0),
                                             (0, -1, 2), (0, 0, 1)])
def test_batch_equals_single_chains(warps, coop, form):
    """CTA size tuned or fixed; the cooperative z-step by the automatic rule,
    off, or taking every document of at least 64 tokens / every document; the
    launch form tuned, one persistent launch per sweep (grid barriers between
    the phases), or six launches."""
    import paper_1704_03581_gb300 as P
    chains = make_chains()
    b = P.Batch(chains, warps_per_block=warps, coop_min_len=coop, batch_form=form)
    b.sweep(4)
    b.sweep(10)           # tuning sweeps (up to 12), then graph replays across two calls
    w, coop_len, tuned, one, layout = b.tuning()
    assert layout in (1, 2)
    assert tuned and w in (2, 4, 8)
    assert coop_len == (coop if coop != 0 else coop_len) and (coop_len == -1 or coop_len >= 1)
    if form == 2:
        assert one
    if form == 1 or coop > 0:
        assert not one
    for i, c in enumerate(chains):
        s = P.Sampler(c["w"], c["doc_off"], c["K"], c["V"], c["alpha"], c["beta"], c["seed"])
        s.sweep(14)
        assert np.array_equal(b.z(i), s.z()), f"chain {i} differs from its single-chain run"
        sb, ss = b.stats(i), s.stats()
        for k in ("tokens", "a_branch", "sum_min", "zero_mass", "dead_rows", "nnz_phi", "sweep",
                  "cum_tokens", "cum_a_branch", "cum_sum_min"):
            assert sb[k] == ss[k], (i, k, sb[k], ss[k])
        s.close()
    b.close()


@pytest.mark.parametrize("n,form", [(3, 2), (3, 1), (4, 2), (4, 1)])
def test_batch_lane_widths(n, form):
    """The batched z-step gives each lane z_lane_topics(largest K) topics: a
    batch of the first three chains (K up to 100: 8 per lane) or four (K up to
    500: 16 per lane), in either launch form, equals each chain run alone
    (whose own lane width follows its own K)."""
    import paper_1704_03581_gb300 as P
    chains = make_chains()[:n]
    b = P.Batch(chains, coop_min_len=-1, batch_form=form)
    b.sweep(5)
    for i, c in enumerate(chains):
        s = P.Sampler(c["w"], c["doc_off"], c["K"], c["V"], c["alpha"], c["beta"], c["seed"], coop_min_len=-1)
        s.sweep(5)
        assert np.array_equal(b.z(i), s.z()), f"chain {i} differs from its single-chain run"
        s.close()
    b.close()


@pytest.mark.parametrize("layout,form", [(1, 2), (2, 2), (2, 1), (0, 2)])
def test_batch_alias_layouts(layout, form):
    """The alias tables as threshold and topic arrays (1), as packed 8-byte
    slots (2), or timed against each other on two sweeps each (0), in the
    one-launch and the six-launch form: every chain equals its single-handle
    run (arrays) and the batch reports the layout it uses."""
    import paper_1704_03581_gb300 as P
    chains = make_chains()
    b = P.Batch(chains, coop_min_len=-1, batch_form=form, alias_layout=layout)
    b.sweep(7)
    w, coop_len, tuned, one, used = b.tuning()
    assert tuned and one == (form == 2)
    assert used == layout if layout else used in (1, 2)
    for i, c in enumerate(chains):
        s = P.Sampler(c["w"], c["doc_off"], c["K"], c["V"], c["alpha"], c["beta"], c["seed"], coop_min_len=-1)
        s.sweep(7)
        assert np.array_equal(b.z(i), s.z()), f"chain {i} differs from its single-chain run"
        s.close()
    b.close()


def test_batch_chain_matches_oracle():
    import paper_1704_03581_gb300 as P
    chains = make_chains()
    b = P.Batch(chains)
    b.sweep(5)
    for i in (1, 3):
        c = chains[i]
        ch = O.Chain(c["w"], c["doc_off"], c["K"], c["V"], c["alpha"], c["beta"], c["seed"]).sweep(5)
        assert np.array_equal(b.z(i), ch.z), f"chain {i} differs from the oracle"
    b.close()


def test_batch_reports_the_failing_chain():
    import paper_1704_03581_gb300 as P
    chains = make_chains()[:3]
    chains[2] = dict(chains[2], V=5)          # word ids beyond V
    with pytest.raises(P.PuldaError) as e:
        P.Batch(chains)
    assert "chain 2" in str(e.value)


def test_grid_barrier_times_out_and_reports():
    """The one-launch form's grid barrier: with every CTA present each of the
    rounds opens; with one CTA short none does, every CTA gives up after its
    2 s limit and the host reads PULDA_ERR_TIMEOUT -- and the device still
    runs a batch afterwards."""
    import time
    import paper_1704_03581_gb300 as P
    st, n = P.pulda_barrier_selftest(64, 0, 5)
    assert st == 0 and n == 64 * 5
    t0 = time.monotonic()
    st, n = P.pulda_barrier_selftest(64, 1, 5)
    dt = time.monotonic() - t0
    assert st == -4 and n == 0 and 1.5 < dt < 30.0
    chains = make_chains()[:3]
    b = P.Batch(chains, coop_min_len=-1, batch_form=2)
    b.sweep(3)
    b.sync()
    b.close()
