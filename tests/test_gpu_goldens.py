"""GPU: Algorithm 1 at the exact-enumeration workloads' own sizes against
FP64 oracle values stored in tests/golden/exact_goldens.json (written by
tests/golden/make_exact_goldens.py, which calls only the oracle).

  * the twelve N = 18 T-doped states (eta in {1, 4, 16} x n_T in
    {0, 8, 32, 64}): sre_exact in FP32 and in split-BF16 x3;
  * sixteen uneven-batch states (N = 9..16): one sre_exact_batched call over
    all of them, and the same call with the states interleaved among
    others of the batch workload.

M_1, M_2, M_3 within 1e-5; nullity and the stabilizer count bit-exact. Each
state is the oracle's FP64 circuit output rounded to complex64, the array the
golden values were computed from (its hash is checked first)."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2601_00761_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_M = 1e-5
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "exact_goldens.json")


def _records(which):
    if not os.path.exists(GOLD):
        pytest.skip("tests/golden/exact_goldens.json has not been written")
    with open(GOLD) as f:
        recs = json.load(f)["states"]
    return [r for r in recs if r["set"] == which]


def _gates(rec):
    if rec["set"] == "n18":
        sp = next(s for s in inputs.workload_n18_gate_lists() if s["seed"] == rec["seed"])
        return sp["gates"]
    sp = inputs.workload_batched_specs(count=4096)[rec["index"]]
    assert sp["seed"] == rec["seed"] and sp["N"] == rec["N"]
    return inputs.batched_gate_list(sp)


def _state(rec):
    psi = oracle.circuit_state(rec["N"], _gates(rec))
    h = hashlib.sha256(np.ascontiguousarray(psi, dtype=np.complex64).tobytes()).hexdigest()[:16]
    assert h == rec["state_sha256_16"], "the oracle's circuit state differs from the one the goldens were made on"
    return torch.from_numpy(psi).cuda()


def _agree(r, rec):
    assert np.max(np.abs(np.array(r["M"]) - np.array(rec["M"]))) < TOL_M, (r["M"], rec["M"])
    # the a-priori FP32 rounding bound the sweep reports holds for every alpha
    for a in range(3):
        assert abs(r["M"][a] - rec["M"][a]) <= r["err_M"][a], (a, r["M"][a], rec["M"][a], r["err_M"][a])
    assert r["nullity"] == rec["nullity"], (r["nullity"], rec["nullity"])
    assert r["stab_count"] == rec["stab_count"], (r["stab_count"], rec["stab_count"])


@pytest.fixture(scope="module")
def sre():
    import paper_2601_00761_gb300 as s
    from paper_2601_00761_gb300 import build
    build.build()
    s.load()
    s.sre_autotune_clear(0)     # the planned tilings, whatever ran before in this process
    return s


@pytest.mark.parametrize("i", range(12))
@pytest.mark.parametrize("precision", [0, 2])   # SRE_FP32_SIMT, SRE_BF16X3_TC
def test_exact_n18_vs_oracle_golden(sre, i, precision):
    recs = _records("n18")
    if i >= len(recs):
        pytest.skip("golden not written for this state")
    rec = recs[i]
    r = sre.sre_exact(_state(rec), allow_nullity_error=True, precision=precision)
    _agree(r, rec)


def test_batched_vs_oracle_golden(sre):
    recs = _records("batched")
    assert len(recs) == 16 and sorted({r["N"] for r in recs}) == list(range(9, 17))
    states = [_state(rec) for rec in recs]
    for r, rec in zip(sre.sre_exact_batched(states), recs):
        _agree(r, rec)
    # the same states interleaved with other states of the workload (other
    # chunk positions, other launch shapes)
    others = []
    for sp in inputs.workload_batched_specs(count=40, seed0=6000):
        p = torch.zeros(1 << sp["N"], dtype=torch.complex64, device="cuda")
        p[0] = 1
        sre.apply_clifford_tdoped_circuit(p, inputs.batched_gate_list(sp))
        others.append(p)
    mixed, where = [], []
    for k, p in enumerate(states):
        mixed.extend(others[2 * k:2 * k + 2])
        where.append(len(mixed))
        mixed.append(p)
    res = sre.sre_exact_batched(mixed)
    for k, rec in zip(where, recs):
        _agree(res[k], rec)
    # every family of every state in one persistent launch (dependency queue)
    res = sre.sre_exact_batched(mixed, batch_queue=1)
    for k, rec in zip(where, recs):
        _agree(res[k], rec)
