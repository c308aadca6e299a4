"""GPU at the N=30 scale of the preconditioned MC workload (3 transform
passes, 8 GiB state): |T>^k |0>^{N-k} prepared on the device, a random
2000-gate {H, S, CNOT} preconditioner applied by the gate kernels, then the
marginal MC. Expected values need no N=30 transform on the host: by Clifford
invariance c_P(C psi) = sign * c_{P'}(psi) with C^dag P C = sign P' (oracle
tableau) and c_{P'} of a product state is a product of one-qubit values; M_2
of the state is k log2(4/3) exactly."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_00761_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, K_T = 30, 12


def _product_c(x, z):
    """c of P_{x,z} on |T>^{K_T} |0>^{N-K_T} (qubit j = bit j)."""
    r2 = 1.0 / math.sqrt(2.0)
    v = 1.0
    for j in range(N):
        a, b = (x >> j) & 1, (z >> j) & 1
        if j < K_T:
            v *= {(0, 0): 1.0, (0, 1): 0.0, (1, 0): r2, (1, 1): r2}[(a, b)]
        else:
            v *= {(0, 0): 1.0, (0, 1): 1.0, (1, 0): 0.0, (1, 1): 0.0}[(a, b)]
        if v == 0.0:
            return 0.0
    return v


@pytest.fixture(scope="module")
def run():
    import paper_2601_00761_gb300 as sre
    from paper_2601_00761_gb300 import build
    build.build()
    sre.load()
    prep = np.array([(inputs.GATE_H, q, 0) for q in range(K_T)] + [(inputs.GATE_T, q, 0) for q in range(K_T)],
                    dtype=np.uint8)
    C = inputs.random_clifford_gates(N, 2000, 30)
    p = torch.zeros(1 << N, dtype=torch.complex64, device="cuda")
    p[0] = 1
    sre.apply_clifford_tdoped_circuit(p, np.concatenate([prep, C]))
    assert abs(sre.sre_norm2(p) - 1.0) < 1e-3
    r = sre.sre_mc(p, sre.SRE_MC_MARGINAL, 48, 16, seed=30, return_samples=True)
    out = {"sre": sre, "C": C, "r": r, "plan": sre.sre_make_plan(N)}
    del p
    torch.cuda.empty_cache()
    return out


def test_n30_runs_three_passes(run):
    assert run["plan"]["n_passes"] == 3 and run["r"]["n_passes"] == 3


def test_n30_sampled_expectations_exact(run):
    r, C = run["r"], run["C"]
    xs = r["xs"].cpu().numpy().astype(np.uint64)
    zs = r["zs"].cpu().numpy().astype(np.uint64)
    c = r["c"].cpu().numpy()
    checked = 0
    for i in range(0, 48, 5):
        for k in range(0, 16, 5):
            x2, z2, sg = oracle.clifford_conjugate(N, C, int(xs[i]), int(zs[i, k]))
            want = sg * _product_c(x2, z2)
            assert abs(c[i, k] - want) < 2e-5, (i, k, c[i, k], want)
            assert want != 0.0          # a drawn string has c^2 > 0
            checked += 1
    assert checked >= 30


def test_n30_m2_clifford_invariant(run):
    r = run["r"]
    want = K_T * math.log2(4.0 / 3.0)
    assert abs(r["M_rb"][1] - want) < 5 * r["err_rb"][1] + 2e-3
    assert abs(r["M_rb"][0] - K_T / 2.0) < 5 * r["err_rb"][0] + 2e-3
