"""The continuous-batching fold-in server: every request's topics equal
pulda_infer on that document alone (and the oracle's fold-in), whatever else
shared the GPU with it -- under memory pressure, few slots and small slices
that split sweeps across launches."""
import threading
import time

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03581_gb300 import build
    build.build()
    import paper_1704_03581_gb300 as P
    from paper_1704_03581_gb300 import synth
    c = synth.tiny()
    s = P.Sampler(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=3).sweep(3)
    ch = O.Chain(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=3).sweep(3)
    yield P, s, ch, c
    s.close()


def requests(c, n, rng):
    out = []
    for i in range(n):
        L = int(rng.choice([1, 2, 31, 32, 33, 100, 257, 500, 3000]))
        out.append(dict(id=1000 + i, seed=int(rng.integers(1, 2 ** 63)), words=rng.integers(0, c.V, L).astype(np.int32),
                        sweeps=int(rng.integers(1, 12))))
    return out


@pytest.mark.parametrize("K", [300, 1000, 1500])
def test_server_lane_widths(trained, K):
    """Models whose K gives the server 16 (K = 300), 32 (K = 1000) and 64
    (K = 1500) topics per lane: every request equals its run alone."""
    P, _, _, c = trained
    s = P.Sampler(c.w, c.doc_off, K, c.V, 0.1, 0.01, seed=4).sweep(2)
    rng = np.random.default_rng(K)
    reqs = requests(c, 16, rng)
    srv = P.Server(s, token_budget=4000, max_slots=8, slice_tokens=64)
    for r in reqs:
        srv.submit(r["id"], r["seed"], r["words"], r["sweeps"])
    got = {}
    t0 = time.time()
    while len(got) < len(reqs):
        for res in srv.poll(timeout_ms=200):
            assert res["status"] == 0
            got[res["req_id"]] = res["z"]
        assert time.time() - t0 < 120, "server made no progress"
    srv.close()
    for r in reqs:
        alone = s.infer(r["words"], np.array([0, len(r["words"])]), r["sweeps"], seed=r["seed"])
        assert np.array_equal(got[r["id"]], alone), f"request {r['id']} differs from its run alone"
    s.close()


@pytest.mark.parametrize("budget,slots,slice_", [(3000, 8, 64), (10000, 64, 4096), (3000, 3, 1), (10000, 64, 0)])
def test_mixed_requests_equal_each_alone(trained, budget, slots, slice_):
    P, s, ch, c = trained
    rng = np.random.default_rng(budget + slots + slice_)
    reqs = requests(c, 40, rng)
    srv = P.Server(s, token_budget=budget, max_slots=slots, slice_tokens=slice_)
    for r in reqs:
        srv.submit(r["id"], r["seed"], r["words"], r["sweeps"])
    got = {}
    t0 = time.time()
    while len(got) < len(reqs):
        for res in srv.poll(timeout_ms=200):
            assert res["status"] == 0
            got[res["req_id"]] = res["z"]
        assert time.time() - t0 < 120, "server made no progress"
    srv.close()
    for r in reqs:
        alone = s.infer(r["words"], np.array([0, len(r["words"])]), r["sweeps"], seed=r["seed"])
        assert np.array_equal(got[r["id"]], alone), f"request {r['id']} differs from its run alone"
    for r in reqs[:5]:
        zo = O.infer(ch.tables, r["words"], np.array([0, len(r["words"])]), r["sweeps"], r["seed"])
        assert np.array_equal(got[r["id"]], zo)


def test_concurrent_submitters_and_bounded_poll(trained):
    P, s, ch, c = trained
    srv = P.Server(s, token_budget=5000, max_slots=16, slice_tokens=256)
    assert srv.poll(timeout_ms=50) == []              # idle: the wait ends with a timeout
    rng = np.random.default_rng(9)
    reqs = requests(c, 60, rng)
    half = len(reqs) // 2

    def submit(part):
        for r in part:
            srv.submit(r["id"], r["seed"], r["words"], r["sweeps"])
    ts = [threading.Thread(target=submit, args=(reqs[:half],)), threading.Thread(target=submit, args=(reqs[half:],))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    got = {}
    t0 = time.time()
    while len(got) < len(reqs) and time.time() - t0 < 120:
        for res in srv.poll(timeout_ms=200):
            got[res["req_id"]] = res["z"]
    srv.close()
    assert len(got) == len(reqs)
    for r in reqs[::7]:
        alone = s.infer(r["words"], np.array([0, len(r["words"])]), r["sweeps"], seed=r["seed"])
        assert np.array_equal(got[r["id"]], alone)


def test_invalid_submissions(trained):
    P, s, ch, c = trained
    srv = P.Server(s, token_budget=100, max_slots=2, slice_tokens=32)
    bad = [(np.zeros(0, np.int32), 1), (np.zeros(101, np.int32), 1), (np.array([c.V], np.int32), 1),
           (np.zeros(5, np.int32), 0)]
    for words, sweeps in bad:
        with pytest.raises(P.PuldaError):
            srv.submit(1, 1, words, sweeps)
    srv.close()


@pytest.mark.parametrize("coop,slice_", [(40, 0), (40, 33), (-1, 0)])
def test_cooperative_requests_equal_each_alone(trained, coop, slice_):
    """Requests of at least `coop` tokens on CTAs of the cooperative z-step while
    the others run one per warp on the second stream; the 2 ms window (slice 0)
    or 33-token slices split their sweeps across launches."""
    P, s0, ch, c = trained
    s = P.Sampler(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=3, coop_min_len=coop).sweep(3)
    rng = np.random.default_rng(7 + coop + slice_)
    reqs = requests(c, 30, rng)
    srv = P.Server(s, token_budget=20000, max_slots=32, slice_tokens=slice_)
    for r in reqs:
        srv.submit(r["id"], r["seed"], r["words"], r["sweeps"])
    got = {}
    t0 = time.time()
    while len(got) < len(reqs):
        for res in srv.poll(timeout_ms=200):
            assert res["status"] == 0
            got[res["req_id"]] = res["z"]
        assert time.time() - t0 < 120, "server made no progress"
    srv.close()
    for r in reqs:
        alone = s0.infer(r["words"], np.array([0, len(r["words"])]), r["sweeps"], seed=r["seed"])
        if not np.array_equal(got[r["id"]], alone):
            zo = O.infer(ch.tables, r["words"], np.array([0, len(r["words"])]), r["sweeps"], r["seed"])
            raise AssertionError(f"request {r['id']} ({len(r['words'])} tokens, {r['sweeps']} sweeps) differs from "
                                 f"its run alone; served == oracle: {np.array_equal(got[r['id']], zo)}, "
                                 f"alone == oracle: {np.array_equal(alone, zo)}")
    for r in reqs[:4]:
        zo = O.infer(ch.tables, r["words"], np.array([0, len(r["words"])]), r["sweeps"], r["seed"])
        assert np.array_equal(got[r["id"]], zo)
    s.close()
