"""The caller's device allocator (pulda_options alloc / free): every device
buffer of a handle, its temporaries, a server and a batch goes through it;
an allocation that fails (injected on the host: the callback returns NULL on
its k-th call, for every k) makes the call return PULDA_ERR_OOM having given
back everything it took, and the next call on a fresh handle works."""
import numpy as np
import pytest

from paper_1704_03581_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03581_gb300 import build
    build.build()


class Ledger:
    """Device memory from torch's caching allocator on one stream, with a
    ledger of what is out and an injected failure at the fail_at-th call."""

    def __init__(self, stream, fail_at: int = 0):
        self.stream, self.fail_at = stream, fail_at
        self.calls = 0
        self.live = {}

    def alloc(self, nbytes, stream):
        import torch
        self.calls += 1
        if self.calls == self.fail_at:
            return 0
        with torch.cuda.stream(self.stream):
            t = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
        assert t.data_ptr() % 256 == 0
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr, stream):
        del self.live[ptr]


def _corpus():
    c = synth.tiny()
    return c.w, c.doc_off, 20, c.V


def test_every_allocation_of_init_can_fail_cleanly():
    import torch
    import paper_1704_03581_gb300 as P
    w, off, K, V = _corpus()
    st = torch.cuda.Stream()
    count = Ledger(st)
    s = P.Sampler(w, off, K, V, 0.1, 0.01, seed=3, stream=st.cuda_stream, allocator=count)
    n_allocs = count.calls
    assert n_allocs >= 20 and len(count.live) == n_allocs
    s.sweep(3)
    z_mine = s.z()
    s.close()
    assert not count.live                       # pulda_free gave everything back
    ref = P.Sampler(w, off, K, V, 0.1, 0.01, seed=3).sweep(3)
    assert np.array_equal(z_mine, ref.z())      # the allocator never changes results
    ref.close()
    for k in range(1, n_allocs + 1):
        led = Ledger(st, fail_at=k)
        with pytest.raises(P.PuldaError) as e:
            P.Sampler(w, off, K, V, 0.1, 0.01, seed=3, stream=st.cuda_stream, allocator=led)
        assert e.value.status == -2, (k, str(e.value))
        assert not led.live, (k, len(led.live))
    again = P.Sampler(w, off, K, V, 0.1, 0.01, seed=3, stream=st.cuda_stream, allocator=Ledger(st))
    again.close()


def test_temporaries_fail_cleanly_and_leave_the_handle_usable():
    import torch
    import paper_1704_03581_gb300 as P
    w, off, K, V = _corpus()
    st = torch.cuda.Stream()
    led = Ledger(st)
    s = P.Sampler(w, off, K, V, 0.1, 0.01, seed=4, stream=st.cuda_stream, allocator=led).sweep(2)
    base = dict(led.live)
    new = synth.tiny().slice_docs(0, 50)
    z_ref = s.infer(new.w, new.doc_off, 3, seed=8, want_m=True)
    calls = {}
    for name, fn in [("infer", lambda: s.infer(new.w, new.doc_off, 3, seed=8, want_m=True)),
                     ("counts", lambda: s.n()), ("m", lambda: s.m()), ("log_posterior", lambda: s.log_posterior()),
                     ("phi", lambda: s.phi())]:
        c0 = led.calls
        fn()
        calls[name] = led.calls - c0
        assert calls[name] >= 1 and led.live.keys() == base.keys(), name
        for k in range(1, calls[name] + 1):
            led.fail_at = led.calls + k
            with pytest.raises(P.PuldaError) as e:
                fn()
            assert e.value.status == -2, (name, k)
            torch.cuda.synchronize()
            assert led.live.keys() == base.keys(), (name, k)
        led.fail_at = 0
    z2, m2 = s.infer(new.w, new.doc_off, 3, seed=8, want_m=True)
    assert np.array_equal(z2, z_ref[0]) and np.array_equal(m2, z_ref[1])
    assert calls["infer"] == 5
    s.close()
    assert not led.live


def test_server_and_batch_take_the_callers_memory():
    import torch
    import paper_1704_03581_gb300 as P
    w, off, K, V = _corpus()
    st = torch.cuda.Stream()
    led = Ledger(st)
    s = P.Sampler(w, off, K, V, 0.1, 0.01, seed=5, stream=st.cuda_stream, allocator=led).sweep(2)
    base = set(led.live)
    c0 = led.calls
    srv = P.Server(s, token_budget=1 << 16, max_slots=64)
    n_srv = led.calls - c0
    assert n_srv == 6
    doc = synth.tiny().w[:120]
    zq = srv.submit(1, 9, doc, 3)
    got = []
    while not got:
        got = srv.poll(timeout_ms=1000)
    srv.close()
    assert set(led.live) == base
    assert np.array_equal(got[0]["z"], s.infer(doc, np.array([0, doc.shape[0]], np.int64), 3, seed=9))
    for k in range(1, n_srv + 1):
        led.fail_at = led.calls + k
        with pytest.raises(P.PuldaError) as e:
            P.Server(s, token_budget=1 << 16, max_slots=64)
        assert e.value.status == -2 and set(led.live) == base, k
    led.fail_at = 0
    s.close()
    assert not led.live
    part = synth.tiny().slice_docs(0, 50)
    chains = [dict(w=w, doc_off=off, K=K, V=V, seed=11), dict(w=part.w, doc_off=part.doc_off, K=7, V=V, seed=12)]
    bl = Ledger(st)
    b = P.Batch(chains, stream=st.cuda_stream, warps_per_block=4, allocator=bl)
    n_b = bl.calls
    b.sweep(3)
    zb = [b.z(i) for i in range(2)]
    b.close()
    assert not bl.live
    ref = P.Batch(chains, warps_per_block=4).sweep(3)
    assert all(np.array_equal(zb[i], ref.z(i)) for i in range(2))
    ref.close()
    for k in range(1, n_b + 1, max(1, n_b // 12)):
        led2 = Ledger(st, fail_at=k)
        with pytest.raises(P.PuldaError) as e:
            P.Batch(chains, stream=st.cuda_stream, warps_per_block=4, allocator=led2)
        assert e.value.status == -2 and not led2.live, k
