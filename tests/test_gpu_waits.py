"""GPU: the bounded device waits. The bulk-copy z sampler waits on mbarriers
for its copies, and the persistent batched sweep waits on device counters for
the items an item depends on; a wait that cannot complete must end by its
bound with SRE_ETIMEOUT reported on the host and the context left usable. The
tests make such waits (an mbarrier expecting more bytes than arrive; a row
item whose strided items never run); nothing faults or hangs."""
import numpy as np
import pytest

import oracle
from paper_2601_00761_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sre():
    import paper_2601_00761_gb300 as s
    from paper_2601_00761_gb300 import build
    build.build()
    s.load()
    return s


def test_bounded_wait_times_out_and_the_context_survives(sre):
    import time
    t = time.perf_counter()
    st = sre.sre_selftest_bounded_wait()
    dt = time.perf_counter() - t
    assert st == sre.SRE_ETIMEOUT
    assert "bounded wait" in sre.sre_last_error()
    assert 0.1 < dt < 30.0
    # the same process keeps working: an MC call through the sampler's waits
    psi = inputs.haar_state(12, 5)
    r = sre.sre_mc(torch.from_numpy(psi).cuda(), sre.SRE_MC_MARGINAL, 8, 8, seed=3, return_samples=True)
    ref = oracle.mc_marginal(psi, 8, 8, 3, 0)
    assert np.array_equal(r["xs"].cpu().numpy().astype(np.uint64), ref["xs"])


def test_queue_wait_times_out_and_the_context_survives(sre):
    """The dependency waits of the persistent batched queue (batch_queue=1):
    one row item whose strided items never run must give up by its bound
    (SRE_ETIMEOUT, about a second of the global timer), and the same process
    then runs a batched sweep through the queue to parity with per-state
    sweeps."""
    import time
    t = time.perf_counter()
    st = sre.sre_selftest_queue_wait()
    dt = time.perf_counter() - t
    assert st == sre.SRE_ETIMEOUT
    assert "queue dependency wait" in sre.sre_last_error()
    assert 0.5 < dt < 30.0
    states = [torch.from_numpy(inputs.haar_state(N, 70 + N)).cuda() for N in (9, 15, 16, 12, 17)]
    res = sre.sre_exact_batched(states, batch_queue=1)
    for p, r in zip(states, res):
        ref = sre.sre_exact(p)
        assert np.max(np.abs(np.array(r["M"]) - np.array(ref["M"]))) < 1e-5
        assert r["nullity"] == ref["nullity"]
