"""GPU parity of the fluctuation ratio r_2 = Std_{x != 0}(m_{2;x}) / E_x[m_{2;x}]
(SM, Clifford preconditioning): exact sweeps against the oracle and the SM's
closed form for |T>^{N/2}|0>^{N/2}; the uniform-x Monte Carlo estimate
against the exact value; and the effect the paper reports, r_2 of the
product magic state collapsing after a random Clifford preconditioner."""
import math

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


def r2_closed(N):
    h = N // 2
    a, b, c = (5 / 4) ** h - 1, 4 ** h - 1, (3 / 2) ** h - 1
    return (8 / 3) ** h * math.sqrt(a / b - c * c / (b * b))


@pytest.mark.parametrize("N", [4, 8, 12, 16])
def test_r2_exact_product_magic_state(sre, N):
    r = sre.sre_exact(dev(inputs.t_product_state(N, N // 2)), allow_nullity_error=True)
    assert abs(r["r2"] - r2_closed(N)) < 1e-5 * r2_closed(N)


@pytest.mark.parametrize("N,seed", [(6, 1), (10, 2), (13, 3)])
def test_r2_exact_vs_oracle(sre, N, seed):
    psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 8 * N, 2, 900 + seed))
    r = sre.sre_exact(dev(psi), allow_nullity_error=True)
    ref = oracle.fluctuation_ratio(psi)
    assert abs(r["r2"] - ref) < 1e-5 * ref + 1e-9


def test_r2_batched_matches_single(sre):
    states = [dev(inputs.t_product_state(10, 5)), dev(inputs.haar_state(12, 4)), dev(inputs.haar_state(10, 5))]
    rs = sre.sre_exact_batched(states)
    for st, rb in zip(states, rs):
        assert abs(rb["r2"] - sre.sre_exact(st, allow_nullity_error=True)["r2"]) < 1e-9 * max(1.0, rb["r2"])


def test_r2_mc_uniform_estimate(sre):
    N = 12
    psi = inputs.haar_state(N, 12)
    exact = sre.sre_exact(dev(psi))["r2"]
    mc = sre.sre_mc(dev(psi), sre.SRE_MC_UNIFORM, 4096, 1, seed=3)["r2"]
    assert abs(mc - exact) < 0.1 * exact


def test_r2_marginal_mode_is_nan(sre):
    r = sre.sre_mc(dev(inputs.haar_state(8, 1)), sre.SRE_MC_MARGINAL, 16, 4, seed=1)
    assert math.isnan(r["r2"])


def test_clifford_preconditioning_reduces_r2(sre):
    """|T>^{N/2}|0>^{N/2} has r_2 ~ (20/9)^{N/4}; a random Clifford circuit
    leaves M_2 unchanged and brings r_2 to order one (main text, Clifford
    preconditioning)."""
    N = 14
    psi = dev(inputs.t_product_state(N, N // 2))
    before = sre.sre_exact(psi, allow_nullity_error=True)
    sre.apply_clifford_tdoped_circuit(psi, inputs.random_clifford_gates(N, 60 * N, 14))
    after = sre.sre_exact(psi, allow_nullity_error=True)
    assert abs(after["M"][1] - before["M"][1]) < 1e-4
    assert before["r2"] > 10.0 and after["r2"] < 2.0
