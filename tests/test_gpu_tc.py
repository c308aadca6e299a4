"""GPU: the split-BF16 tensor-core form of the family transform (H_16
Kronecker factors on mma.sync BF16 -> FP32) against the FP64 oracle.

Tolerance of the three-way split (BF16X3): |dc| <= 5e-6 per Pauli expectation,
|dM| <= 1e-5. The two-way split (BF16X2) keeps about 16 mantissa bits per
stage; its error is measured and bounded loosely (it is not the accurate form)."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_00761_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_TC = 5e-6
TOL_M = 1e-5
BF16X2, BF16X3 = 1, 2


@pytest.fixture(scope="module")
def sre():
    import paper_2601_00761_gb300 as s
    from paper_2601_00761_gb300 import build
    build.build()
    s.load()
    return s


def dev(psi):
    return torch.from_numpy(np.ascontiguousarray(psi, dtype=np.complex64)).cuda()


@pytest.mark.parametrize("N", [11, 13, 15, 18, 24])
def test_tc_bf16x3_spectrum(sre, N):
    psi = inputs.haar_state(N, 900 + N)
    p = dev(psi)
    worst = 0.0
    for x in (0, 1, (1 << N) - 1, (1 << (N - 1)) | 3):
        c = sre.sre_family_spectrum(p, x, precision=BF16X3).cpu().numpy()
        worst = max(worst, float(np.max(np.abs(c - oracle.family_spectrum(psi, x)))))
    assert worst < TOL_TC, worst


@pytest.mark.parametrize("N", [12, 18])
def test_tc_bf16x3_large_coefficients(sre, N):
    """|c| near 1 (stabilizer-like families) is where a split loses most."""
    gates = inputs.random_clifford_tdoped_gates(N, 6 * N, 6, 123 + N)
    psi = oracle.circuit_state(N, gates)
    p = dev(psi)
    for x in (0, 5, (1 << N) - 7):
        c = sre.sre_family_spectrum(p, x, precision=BF16X3).cpu().numpy()
        ref = oracle.family_spectrum(psi, x)
        assert np.max(np.abs(c - ref)) < TOL_TC


def test_tc_bf16x2_error_is_bounded(sre):
    N = 16
    psi = inputs.haar_state(N, 5)
    p = dev(psi)
    c2 = sre.sre_family_spectrum(p, 77, precision=BF16X2).cpu().numpy()
    c3 = sre.sre_family_spectrum(p, 77, precision=BF16X3).cpu().numpy()
    ref = oracle.family_spectrum(psi, 77)
    e2, e3 = np.max(np.abs(c2 - ref)), np.max(np.abs(c3 - ref))
    assert e3 < TOL_TC and e2 < 1e-3 and e3 <= e2


@pytest.mark.parametrize("N,k", [(12, 5), (16, 8)])
def test_tc_exact_closed_form(sre, N, k):
    r = sre.sre_exact(dev(inputs.t_product_state(N, k)), precision=BF16X3)
    assert abs(r["M"][1] - k * math.log2(4 / 3)) < TOL_M
    assert abs(r["M"][0] - k / 2) < TOL_M and r["nullity"] == k


def test_tc_exact_vs_oracle(sre):
    N = 12
    psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 72, 3, 55))
    r = sre.sre_exact(dev(psi), precision=BF16X3, allow_nullity_error=True)
    ref = oracle.sre_exact(psi)
    assert np.max(np.abs(np.array(r["M"]) - ref["M"])) < TOL_M
    assert r["nullity"] == ref["nullity"]


def test_tc_mc_marginal_vs_oracle(sre):
    N = 14
    psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 8 * N, 3, 714))
    r = sre.sre_mc(dev(psi), sre.SRE_MC_MARGINAL, 8, 8, seed=21, return_samples=True, precision=BF16X3)
    ref = oracle.mc_marginal(psi, 8, 8, 21, 0)
    assert np.array_equal(r["xs"].cpu().numpy().astype(np.uint64), ref["xs"])
    assert np.array_equal(r["zs"].cpu().numpy().astype(np.uint64), ref["zs"])
    assert np.max(np.abs(r["c"].cpu().numpy() - ref["c"])) < TOL_TC
    assert np.max(np.abs(np.array(r["M_rb"]) - ref["M_rb"])) < TOL_M
