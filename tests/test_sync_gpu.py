"""Host waits that give up: pulda_sync_timeout returns PULDA_ERR_TIMEOUT while
queued sweeps still run, leaves them running, and a later wait sees them
finish with the same topics as an uninterrupted run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03581_gb300 import build
    build.build()


def test_timeout_then_completion():
    import paper_1704_03581_gb300 as P
    from paper_1704_03581_gb300 import synth
    c = synth.small()
    a = P.Sampler(c.w, c.doc_off, 100, c.V, 0.1, 0.01, seed=11)
    a.sync()
    P.pulda_sweep(a.h, 60)                       # queued, hundreds of ms of work
    assert P.pulda_sync_timeout(a.h, 0) is False
    assert P.pulda_sync_timeout(a.h, 120000) is True
    b = P.Sampler(c.w, c.doc_off, 100, c.V, 0.1, 0.01, seed=11).sweep(60)
    assert np.array_equal(a.z(), b.z())
    with pytest.raises(P.PuldaError):
        P.pulda_sync_timeout(a.h, -1)
    a.close()
    b.close()
