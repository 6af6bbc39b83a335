"""Cases run against the checked build (PULDA_LIB pointing at it) by
test_checked_gpu.py in a process of their own: the one-warp, grouped and
cooperative z-steps, fold-in, the batched form and the server, each compared
with the oracle or with its single-chain run; any bounds error a kernel
raises surfaces as a PuldaError from the next sync."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_1704_03581_gb300 as P  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1704_03581_gb300 import synth  # noqa: E402
from parity_util import first_mismatch, lockstep  # noqa: E402


def corpus(rng, lengths, V):
    off = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    p = (1.0 + np.arange(V)) ** -1.0
    return rng.choice(V, size=int(off[-1]), p=p / p.sum()).astype(np.int32), off


def main():
    assert os.path.realpath(P.LIB_PATH).endswith(os.path.join("_build_checked", "libpulda.so")), P.LIB_PATH
    c = synth.tiny()
    for path in (0, 1, 2):
        for coop in (-1, 1):
            s, _ = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=path, sweeps=2, path=path, coop_min_len=coop)
            s.close()
    s, _ = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=4, sweeps=2, docs_per_warp=4)
    s.close()
    rng = np.random.default_rng(9)
    for K in (1, 33, 300, 1000, 1025):
        lengths = rng.integers(0, 400, size=30)
        lengths[:3] = [0, 1, 1500]
        w, off = corpus(rng, lengths, 600)
        for coop in (-1, 200):
            s, _ = lockstep(w, off, K, 600, 0.2, 0.02, seed=K, sweeps=2, coop_min_len=coop)
            s.close()
    s, ch = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=2, sweeps=2, coop_min_len=50)
    new = c.slice_docs(0, 40)
    assert not first_mismatch(s.infer(new.w, new.doc_off, 5, seed=3), O.infer(ch.tables, new.w, new.doc_off, 5, 3),
                              new.doc_off)
    srv = P.Server(s, token_budget=20000, max_slots=16, slice_tokens=0)
    reqs = [(100 + i, rng.integers(0, c.V, int(n)).astype(np.int32)) for i, n in enumerate([3, 64, 900, 40, 1200])]
    for rid, words in reqs:
        srv.submit(rid, rid, words, 4)
    got = {}
    while len(got) < len(reqs):
        for r in srv.poll(timeout_ms=500):
            assert r["status"] == 0
            got[r["req_id"]] = r["z"]
    srv.close()
    for rid, words in reqs:
        assert np.array_equal(got[rid], s.infer(words, np.array([0, len(words)]), 4, seed=rid))
    s.close()
    chains = []
    for i, (K, V, D, mean) in enumerate([(37, 300, 80, 60), (500, 900, 40, 700)]):
        lengths = rng.poisson(mean, size=D)
        w, off = corpus(rng, lengths, V)
        chains.append(dict(w=w, doc_off=off, K=K, V=V, alpha=0.1, beta=0.01, seed=50 + i))
    b = P.Batch(chains, coop_min_len=300)
    b.sweep(3)
    for i, cc in enumerate(chains):
        one = P.Sampler(cc["w"], cc["doc_off"], cc["K"], cc["V"], 0.1, 0.01, cc["seed"]).sweep(3)
        assert np.array_equal(b.z(i), one.z())
        one.close()
    b.close()
    print("checked build: all cases passed")


if __name__ == "__main__":
    main()
