"""GPU parity of the mixed-state SRE (SM, "Stabilizer Renyi entropy of mixed
states", Eq. Msre-mixed): sre_mixed against the FP64 oracle (the SM's
partial-sum route, itself pinned to the definition) and the closed forms of
product states, Bell pairs and GHZ states."""
import math

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


def dev(psi):
    return torch.from_numpy(np.ascontiguousarray(psi, dtype=np.complex64)).cuda()


@pytest.mark.parametrize("N,NA", [(1, 1), (2, 1), (5, 2), (8, 3), (10, 10), (12, 6), (14, 9), (15, 12)])
def test_mixed_vs_oracle(sre, N, NA):
    psi = inputs.unnormalised_gaussian_state(N, 300 + N + NA)
    r = sre.sre_mixed(dev(psi), NA)
    ref = oracle.sre_mixed(psi, NA)
    assert abs(r["S2"] - ref["S2"]) < TOL_M
    assert np.max(np.abs(np.array(r["M"][1:]) - ref["M"][1:])) < TOL_M
    assert np.allclose(r["W"][:3], ref["W"][:3], rtol=1e-5)


@pytest.mark.parametrize("N", [12, 15])
def test_mixed_full_subsystem_matches_pure(sre, N):
    psi = dev(inputs.haar_state(N, N))
    r = sre.sre_mixed(psi, N)
    p = sre.sre_exact(psi)
    assert abs(r["S2"]) < 1e-5
    assert np.max(np.abs(np.array(r["M"]) - np.array(p["M"]))) < TOL_M


def test_mixed_product_state(sre):
    NA, NB = 6, 8
    t = inputs.t_product_state(NA, NA).astype(np.complex128)
    b = inputs.haar_state(NB, 7).astype(np.complex128)
    r = sre.sre_mixed(dev(np.kron(b, t)), NA)
    assert abs(r["S2"]) < 1e-5
    assert abs(r["M"][1] - NA * math.log2(4 / 3)) < TOL_M
    assert abs(r["M"][2] - NA * 0.5 * math.log2(8 / 5)) < TOL_M
    assert abs(r["M"][0] - NA * 0.5) < TOL_M    # one |T>: M_1 = 1/2


def test_mixed_bell_pairs_and_ghz(sre):
    NA = 7
    N = 2 * NA
    psi = np.zeros(1 << N, dtype=np.complex64)
    for a in range(1 << NA):
        psi[a | (a << NA)] = 1.0
    r = sre.sre_mixed(dev(psi), NA)
    assert abs(r["S2"] - NA) < TOL_M and abs(r["M"][1]) < TOL_M and abs(r["M"][2] + NA / 2) < TOL_M
    assert math.isnan(r["M"][0])
    g = np.zeros(1 << 16, dtype=np.complex64)
    g[0] = g[-1] = 1.0
    r = sre.sre_mixed(dev(g), 9)
    assert abs(r["S2"] - 1.0) < TOL_M and abs(r["M"][1]) < TOL_M


def test_mixed_n18_sampled_against_oracle(sre):
    N, NA = 18, 9
    psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 6 * N, 3, 18))
    r = sre.sre_mixed(dev(psi), NA)
    ref = oracle.sre_mixed(psi, NA)
    assert np.max(np.abs(np.array(r["M"][1:]) - ref["M"][1:])) < TOL_M and abs(r["S2"] - ref["S2"]) < TOL_M


def test_mixed_gram_tiles_vs_oracle(sre):
    """d_A = 1024: an 8 x 8 grid of 128 x 128 Gram tiles on the tensor cores
    (36 computed, the rest written as conjugate transposes), 8 K blocks."""
    N, NA = 18, 10
    psi = inputs.unnormalised_gaussian_state(N, 1810)
    r = sre.sre_mixed(dev(psi), NA)
    ref = oracle.sre_mixed(psi, NA)
    assert abs(r["S2"] - ref["S2"]) < TOL_M
    assert np.max(np.abs(np.array(r["M"][1:]) - ref["M"][1:])) < TOL_M
    assert np.allclose(r["W"][:3], ref["W"][:3], rtol=1e-5)


def test_mixed_gram_chunked_k(sre):
    """N = 28, N_A = 7: the split planes hold 2^20 of the 2^21 columns of
    Psi, so the Gram matrix is accumulated over two chunks. A product state
    |T>^7 (x) (Haar on 21 qubits) has rho_A pure (S_2 = 0) with M_2 =
    7 log2(4/3), and the GHZ state has rho_A = (|0><0| + |1..1><1..1|)/2
    (S_2 = 1, M_2 = 0)."""
    N, NA = 28, 7
    a = torch.from_numpy(inputs.t_product_state(NA, NA)).cuda()
    b = torch.from_numpy(inputs.haar_state(N - NA, 28)).cuda()
    psi = (b[:, None] * a[None, :]).reshape(-1).contiguous()      # index a + 2^NA e
    r = sre.sre_mixed(psi, NA)
    assert abs(r["S2"]) < 1e-5
    assert abs(r["M"][1] - NA * math.log2(4 / 3)) < TOL_M
    del psi, b
    g = torch.zeros(1 << N, dtype=torch.complex64, device="cuda")
    g[0] = g[-1] = 1.0
    r = sre.sre_mixed(g, NA)
    assert abs(r["S2"] - 1.0) < TOL_M and abs(r["M"][1]) < TOL_M
