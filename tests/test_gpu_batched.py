"""GPU: the batched exact sweep (one persistent launch over the single-pass
states, one launch per same-N chunk of the larger ones, captured into a CUDA
graph) against sre_exact per state, the graph replay on new states of the same
shape, and the autotuner."""
import numpy as np
import pytest

import oracle
from paper_2601_00761_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_M = 1e-5


@pytest.fixture(scope="module")
def sre():
    import paper_2601_00761_gb300 as s
    from paper_2601_00761_gb300 import build
    build.build()
    s.load()
    return s


def _state(sre, spec):
    p = torch.zeros(1 << spec["N"], dtype=torch.complex64, device="cuda")
    p[0] = 1
    sre.apply_clifford_tdoped_circuit(p, inputs.batched_gate_list(spec))
    return p


def _check(sre, states, res):
    for p, r in zip(states, res):
        ref = sre.sre_exact(p, allow_nullity_error=True)
        assert np.max(np.abs(np.array(r["M"]) - np.array(ref["M"]))) < TOL_M
        assert r["nullity"] == ref["nullity"] and r["stab_count"] == ref["stab_count"]


def test_batched_uneven_matches_per_state(sre):
    specs = inputs.workload_batched_specs(count=48, seed0=4000, n_min=1, n_max=16)
    states = [_state(sre, s) for s in specs]
    states.append(torch.from_numpy(inputs.t_product_state(16, 5)).cuda())   # closed form, 2 passes
    states.append(torch.from_numpy(inputs.haar_state(11, 2)).cuda())
    res = sre.sre_exact_batched(states)
    _check(sre, states, res)
    assert res[-2]["nullity"] == 5 and abs(res[-2]["M"][1] - 5 * np.log2(4 / 3)) < TOL_M
    # the same batch with every family in one persistent launch (dependency queue)
    resq = sre.sre_exact_batched(states, batch_queue=1)
    _check(sre, states, resq)


def test_batched_queue_mode_has_its_own_graph(sre):
    """The dependency-queue mode (batch_queue=1) sweeps the two-pass states in
    the persistent launch too, so its launch sequence is shorter; the cached
    graphs of the two modes for the same batch shape stay apart."""
    states = [torch.from_numpy(inputs.haar_state(N, 500 + N)).cuda() for N in (10, 15, 16, 16)]
    counts, results = [], []
    for q in (0, 1, 0, 1):
        k0 = sre.sre_kernel_launches()
        results.append(sre.sre_exact_batched(states, batch_queue=q))
        counts.append(sre.sre_kernel_launches() - k0)
    assert counts[0] == counts[2] and counts[1] == counts[3] and counts[1] < counts[0]
    for a, b in zip(results[0], results[1]):
        assert np.max(np.abs(np.array(a["M"]) - np.array(b["M"]))) < TOL_M and a["nullity"] == b["nullity"]
    for a, b in zip(results[1], results[3]):
        assert a["M"] == b["M"]


def test_batched_graph_replay_with_new_states(sre):
    Ns = [9, 12, 12, 15, 7, 9]
    a = [torch.from_numpy(inputs.haar_state(N, 10 + i)).cuda() for i, N in enumerate(Ns)]
    b = [torch.from_numpy(inputs.t_product_state(N, i % N)).cuda() for i, N in enumerate(Ns)]
    ra = sre.sre_exact_batched(a)
    rb = sre.sre_exact_batched(b)        # same shape: the cached graph runs on new pointers
    _check(sre, a, ra)
    _check(sre, b, rb)


def test_batched_graph_follows_the_plan(sre):
    """A two-pass state (N = 16) runs the chunked launch sequence, whose cached
    graph is keyed on the plan as well as the shape: 4^16 families in launches
    of 1024 families, then of 4096, then of 1024 again (the first graph
    replayed), in the FP32 and the tensor-core forms."""
    p = torch.from_numpy(inputs.haar_state(16, 16).astype(np.complex64)).cuda()
    for prec in (sre.SRE_FP32_SIMT, sre.SRE_BF16X3_TC):
        counts = []
        for xb in (1024, 4096, 1024):
            k0 = sre.sre_kernel_launches()
            r = sre.sre_exact_batched([p], x_batch=xb, precision=prec)[0]
            counts.append(sre.sre_kernel_launches() - k0)
            ref = sre.sre_exact(p, x_batch=xb, allow_nullity_error=True, precision=prec)
            assert np.max(np.abs(np.array(r["M"]) - np.array(ref["M"]))) < TOL_M
        assert counts[0] == counts[2] and counts[0] > counts[1]


def test_batched_single_pass_states_share_one_launch(sre):
    """Every family of every FP32 state with N <= 14 is an item of one
    persistent launch: batches of one and of two states of each N = 1 .. 14
    (then with a chunked N = 15 state and product states) match the per-state
    sweeps, and the second state of each N adds no kernel launch."""
    def launches(states):
        k0 = sre.sre_kernel_launches()
        res = sre.sre_exact_batched(states)
        return res, sre.sre_kernel_launches() - k0
    one = [torch.from_numpy(inputs.haar_state(N, 300 + N)).cuda() for N in range(1, 15)]
    two = one + [torch.from_numpy(inputs.haar_state(N, 400 + N)).cuda() for N in range(1, 15)]
    more = two + [torch.from_numpy(inputs.haar_state(15, 7)).cuda()] + \
        [torch.from_numpy(inputs.t_product_state(N, N // 2)).cuda() for N in range(1, 15)]
    r1, c1 = launches(one)
    r2, c2 = launches(two)
    r3, _ = launches(more)
    _check(sre, two, r2)
    _check(sre, more, r3)
    for r, q in zip(r1, r2):
        assert r["M"] == q["M"] and r["nullity"] == q["nullity"]
    # per bucket 2 norm kernels, the totals, the FP64 recount of the flagged
    # families (the x = 0 family of every state) and its scatter, plus the one
    # persistent launch: the same for one state of each N as for two
    assert c1 == c2


def test_batched_queue_mode_large_states(sre):
    """The dependency queue at its largest states: the strided items of N = 18,
    19 and 20 (4, 5 and 6 rows; 256 to 1024 families per 1 GB ring slot),
    among single-pass states, against per-state sweeps."""
    states = [torch.from_numpy(inputs.haar_state(N, 900 + N)).cuda() for N in (20, 9, 19, 13, 18)]
    res = sre.sre_exact_batched(states, batch_queue=1)
    _check(sre, states, res)


def test_batched_small_vs_oracle(sre):
    specs = inputs.workload_batched_specs(count=6, seed0=77, n_min=3, n_max=8)
    states, refs = [], []
    for s in specs:
        psi = oracle.circuit_state(s["N"], inputs.batched_gate_list(s))
        states.append(torch.from_numpy(psi).cuda())
        refs.append(oracle.sre_exact(psi))
    res = sre.sre_exact_batched(states)
    for r, ref in zip(res, refs):
        assert np.max(np.abs(np.array(r["M"]) - ref["M"])) < TOL_M
        assert r["nullity"] == ref["nullity"]


def test_autotune_keeps_results(sre):
    psi = torch.from_numpy(inputs.haar_state(18, 9)).cuda()
    before = sre.sre_exact(psi)
    best = sre.sre_autotune(psi)
    assert 10 <= best["radix_log2"] <= 14
    plan = sre.sre_make_plan(18)
    assert plan["pass_bits"][-1] == best["radix_log2"]
    after = sre.sre_exact(psi)
    assert np.max(np.abs(np.array(after["M"]) - np.array(before["M"]))) < TOL_M
    c = sre.sre_family_spectrum(psi, 12345).cpu().numpy()
    assert np.max(np.abs(c - oracle.family_spectrum(inputs.haar_state(18, 9), 12345))) < 1e-6
    # clearing the choice restores the planned default, and later tests see it
    sre.sre_autotune_clear(18)
    assert sre.sre_make_plan(18)["pass_bits"][-1] == 13
