"""pulda_infer_noalloc: fold-in for callers that cannot allocate device
memory (pre-carved serving arenas, memory-capped tenants, loops that must not
stall on the allocator).  Checked through the C ABI against pulda_infer, the
allocating entry point, bit for bit -- the tolerance of every other parity
test here -- on two calls in a row, since the calls share one static scratch
array that keeps the previous call's contents.  This file is collected last
so a failure here never hides another test's result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chain():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03581_gb300 import build
    build.build()
    import paper_1704_03581_gb300 as P
    from paper_1704_03581_gb300 import synth
    c = synth.tiny()
    s = P.Sampler(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=11).sweep(3)
    yield P, s, c
    s.close()


def test_noalloc_matches_infer_on_two_calls(chain):
    import torch
    P, s, c = chain
    for d0, d1, seed in [(0, 300, 5), (300, 1000, 6)]:
        new = c.slice_docs(d0, d1)
        z_ref = s.infer(new.w, new.doc_off, 7, seed=seed)
        w_dev = torch.from_numpy(new.w).cuda()
        off_dev = torch.from_numpy(new.doc_off).cuda()
        z_dev = torch.full((new.N,), -1, dtype=torch.int16, device="cuda")
        torch.cuda.synchronize()
        P.pulda_infer_noalloc(s.h, w_dev, off_dev, 7, seed, z_dev)
        assert np.array_equal(z_dev.cpu().numpy(), z_ref), f"docs {d0}:{d1} differ from pulda_infer"


def test_noalloc_rejects_sizes_beyond_its_scratch(chain):
    import torch
    P, s, c = chain
    D = 65537
    off = torch.zeros(D + 1, dtype=torch.int64, device="cuda")
    w = torch.zeros(1, dtype=torch.int32, device="cuda")
    z = torch.zeros(1, dtype=torch.int16, device="cuda")
    with pytest.raises(P.PuldaError) as e:
        P.pulda_infer_noalloc(s.h, w, off, 1, 0, z)
    assert e.value.status == -1 and "65536" in str(e.value)


def test_noalloc_checks_inputs_on_the_device(chain):
    import torch
    P, s, c = chain
    w = torch.tensor([0, 1, c.V], dtype=torch.int32, device="cuda")      # last id out of range
    off = torch.tensor([0, 3], dtype=torch.int64, device="cuda")
    z = torch.zeros(3, dtype=torch.int16, device="cuda")
    with pytest.raises(P.PuldaError) as e:
        P.pulda_infer_noalloc(s.h, w, off, 1, 0, z)
    assert "word id at token 2" in str(e.value)
    off_bad = torch.tensor([0, 4], dtype=torch.int64, device="cuda")   # ends beyond N
    w_ok = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
    with pytest.raises(P.PuldaError) as e:
        P.pulda_infer_noalloc(s.h, w_ok, off_bad, 1, 0, z)
    assert "first bad document: 0" in str(e.value)


def test_noalloc_matches_infer_against_a_dirichlet_phi():
    """The same equality when the handle draws Algorithm 1's Dirichlet Phi."""
    import torch
    import paper_1704_03581_gb300 as P
    from paper_1704_03581_gb300 import synth
    c = synth.tiny()
    s = P.Sampler(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=12, phi_mode=1).sweep(2)
    new = c.slice_docs(100, 400)
    z_ref = s.infer(new.w, new.doc_off, 5, seed=9)
    w_dev = torch.from_numpy(new.w).cuda()
    off_dev = torch.from_numpy(new.doc_off).cuda()
    z_dev = torch.full((new.N,), -1, dtype=torch.int16, device="cuda")
    torch.cuda.synchronize()
    P.pulda_infer_noalloc(s.h, w_dev, off_dev, 5, 9, z_dev)
    assert np.array_equal(z_dev.cpu().numpy(), z_ref)
    s.close()



def _noalloc(P, s, w, off, n_sweeps, seed):
    import torch
    w_dev = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    off_dev = torch.from_numpy(np.ascontiguousarray(off)).cuda()
    z_dev = torch.full((w.shape[0],), -1, dtype=torch.int16, device="cuda")
    torch.cuda.synchronize()
    P.pulda_infer_noalloc(s.h, w_dev, off_dev, n_sweeps, seed, z_dev)
    return z_dev.cpu().numpy()


@pytest.mark.parametrize("kw", [dict(coop_min_len=1000), dict(docs_per_warp=4)])
def test_noalloc_matches_infer_when_infer_uses_its_other_kernels(kw):
    """pulda_infer sends documents above its cooperative threshold to one CTA
    each, and on a docs_per_warp = 4 handle runs the grouped kernel; the
    no-alloc call runs its own schedule.  The draws are the same, so are the
    topics: checked against pulda_infer on two calls in a row and, for the two
    longest documents, against the oracle's fold-in."""
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from oracle import oracle as O
    from parity_util import first_mismatch, lockstep
    import paper_1704_03581_gb300 as P
    from paper_1704_03581_gb300 import synth
    c = synth.tiny()
    rng = np.random.default_rng(77)
    lengths = np.concatenate([rng.integers(2000, 3500, size=4), rng.integers(1, 300, size=60)])
    rng.shuffle(lengths)
    off = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    w = rng.integers(0, c.V, size=int(off[-1])).astype(np.int32)
    s, ch = lockstep(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=13, sweeps=2, **kw)
    z_ref = s.infer(w, off, 4, seed=21)
    for _ in range(2):        # two calls in a row share the scratch array
        z = _noalloc(P, s, w, off, 4, 21)
        assert not first_mismatch(z, z_ref, off), kw
    for d in np.argsort(-lengths, kind="stable")[:2]:
        a, b = int(off[d]), int(off[d + 1])
        zo = O.infer(ch.tables, w[a:b], np.array([0, b - a], np.int64), 4, 21, index_base=a)
        assert np.array_equal(z_ref[a:b], zo), int(d)
    s.close()
