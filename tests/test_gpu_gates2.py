"""GPU parity of the general two-qubit gates (brick-wall circuits of the
Supplemental Material): FP32 states against the FP64 oracle after Haar-random
brick walls and arbitrary ordered pairs; the paper's preconditioner (a random
brick-wall Clifford circuit of depth N_C = 2N) leaves M_2 unchanged and
brings r_2 of the product magic state to order one."""
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


def dev(psi):
    return torch.from_numpy(np.ascontiguousarray(psi, dtype=np.complex64)).cuda()


def assert_gate_error(d, ref, n_gates):
    """Per amplitude the 1e-6 target; in l2 norm the FP32 rounding bound of a
    general two-qubit gate: each output is a 4-term complex dot product of a
    unit-norm matrix row with the amplitude quartet (8 real products, error
    <= 8 sqrt2 u |v| per output, 4 outputs) plus the FP32 rounding of the
    matrix itself, under 25 u |psi| per gate."""
    assert np.max(np.abs(d)) < 1e-6
    assert np.linalg.norm(d) <= 25 * 2.0**-24 * n_gates * np.linalg.norm(ref) + 1e-12


@pytest.mark.parametrize("N,depth", [(2, 3), (5, 6), (9, 8), (13, 6), (17, 4)])
def test_brickwall_haar_vs_oracle(sre, N, depth):
    psi = inputs.haar_state(N, 40 + N)
    m, p = inputs.brickwall_circuit(N, depth, "haar", 50 + N)
    g = np.random.default_rng(N)
    extra_m = np.stack([inputs.haar_two_qubit(g) for _ in range(6)]).astype(np.complex64)
    extra_p = []
    for _ in range(6):
        a, b = g.choice(N, 2, replace=False)
        extra_p.append((int(a), int(b)))
    m = np.concatenate([m, extra_m]) if len(m) else extra_m
    p = np.concatenate([p, np.asarray(extra_p, np.int32)]) if len(p) else np.asarray(extra_p, np.int32)
    x = dev(psi)
    sre.apply_two_qubit_gates(x, m, p)
    ref = oracle.apply_two_qubit(psi, m, p)
    assert_gate_error(x.cpu().numpy() - ref, ref, len(p))


def test_brickwall_clifford_on_basis_state_is_a_stabilizer_state(sre):
    N = 12
    m, p = inputs.brickwall_circuit(N, 2 * N, "clifford", 3)
    x = dev(inputs.basis_state(N, 0))
    sre.apply_two_qubit_gates(x, m, p)
    r = sre.sre_exact(x)
    assert r["nullity"] == 0 and abs(r["M"][1]) < 1e-4


def test_brickwall_preconditioner_r2(sre):
    """Main text, Clifford preconditioning: N_C = 2N brick-wall Clifford
    layers leave M_2 = N_T log2(4/3) and reduce r_2 from ~(20/9)^{N/4} to
    order one."""
    N = 16
    x = dev(inputs.t_product_state(N, N // 2))
    before = sre.sre_exact(x, allow_nullity_error=True)
    m, p = inputs.brickwall_circuit(N, 2 * N, "clifford", 16)
    sre.apply_two_qubit_gates(x, m, p)
    after = sre.sre_exact(x, allow_nullity_error=True)
    assert abs(after["M"][1] - (N // 2) * np.log2(4 / 3)) < 1e-4
    assert before["r2"] > 20.0 and after["r2"] < 2.0


def test_many_two_qubit_gates_on_few_qubits(sre):
    """More two-qubit gates than one pass holds matrices for (N = 6: every
    gate fits one 13-qubit block, so the planner splits the list by count)."""
    N = 6
    g = np.random.default_rng(66)
    m = np.stack([inputs.haar_two_qubit(g) for _ in range(1300)]).astype(np.complex64)
    p = np.asarray([tuple(int(v) for v in g.choice(N, 2, replace=False)) for _ in range(1300)], np.int32)
    psi = inputs.haar_state(N, 6)
    x = dev(psi)
    sre.apply_two_qubit_gates(x, m, p)
    ref = oracle.apply_two_qubit(psi, m, p)
    assert_gate_error(x.cpu().numpy() - ref, ref, len(p))
