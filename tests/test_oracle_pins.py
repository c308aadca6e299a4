"""Pins of the FP64 oracle against facts other than itself: closed forms the
paper prints or derives, invariants, special cases that reduce to a library
routine (numpy's Philox, dense Kronecker matrices), and brute force on tiny
inputs. Each plausible mistake planted in the oracle (see test_mutations)
fails at least one of these."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2601_00761_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


# ------------------------------------------------------------------ Philox
@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((123, 456), (7, 8, 9, 10)),
                                     ((2**64 - 1, 1), (2**64 - 2, 5, 0, 0)),
                                     ((0xDEADBEEF, 0), (41, 0, 3, 2**63))])
def test_philox_matches_numpy(key, ctr):
    """numpy's Philox (4x64-10) generates block(counter + 1) first."""
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    ref = g.random_raw(4)
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64
    if ctr[0] == 2**64 - 1:
        c[1] += 1
    assert np.array_equal(oracle.philox4x64_10(c, key), ref)


def test_u01_range():
    assert oracle.u01(0) == 0.0
    assert oracle.u01(2**64 - 1) == 1.0 - 2.0**-53
    assert oracle.u01(1 << 63) == 0.5


# ------------------------------------------------- single-qubit closed forms
def _bloch(a0, a1):
    """<I>, <Z>, <X>, <Y> of a one-qubit state from its amplitudes."""
    n = abs(a0) ** 2 + abs(a1) ** 2
    a0, a1 = a0 / np.sqrt(n), a1 / np.sqrt(n)
    X = 2 * (np.conj(a0) * a1).real
    Y = 2 * (np.conj(a0) * a1).imag
    Z = abs(a0) ** 2 - abs(a1) ** 2
    return {(0, 0): 1.0, (0, 1): Z, (1, 0): X, (1, 1): Y}


ONE_QUBIT = {"0": (1, 0), "1": (0, 1), "+": (1 / np.sqrt(2), 1 / np.sqrt(2)),
             "-": (1 / np.sqrt(2), -1 / np.sqrt(2)), "+i": (1 / np.sqrt(2), 1j / np.sqrt(2)),
             "T": inputs.T_QUBIT}
EXPECTED_ONE_QUBIT = {  # (x, z) -> c: I=(0,0), Z=(0,1), X=(1,0), Y=(1,1)
    "0": {(0, 0): 1, (0, 1): 1, (1, 0): 0, (1, 1): 0},
    "1": {(0, 0): 1, (0, 1): -1, (1, 0): 0, (1, 1): 0},
    "+": {(0, 0): 1, (0, 1): 0, (1, 0): 1, (1, 1): 0},
    "-": {(0, 0): 1, (0, 1): 0, (1, 0): -1, (1, 1): 0},
    "+i": {(0, 0): 1, (0, 1): 0, (1, 0): 0, (1, 1): 1},
    "T": {(0, 0): 1, (0, 1): 0, (1, 0): 1 / np.sqrt(2), (1, 1): 1 / np.sqrt(2)},
}


@pytest.mark.parametrize("name", list(ONE_QUBIT))
def test_single_qubit_expectations(name):
    psi = np.array(ONE_QUBIT[name], dtype=np.complex64)
    for (x, z), want in EXPECTED_ONE_QUBIT[name].items():
        assert abs(oracle.pauli_expectation(psi, x, z) - want) < 1e-7
        assert abs(oracle.family_spectrum(psi, x)[z] - want) < 1e-7


def test_product_state_factorises():
    """c_{x,z} of a product state is the product of one-qubit expectations."""
    g = np.random.default_rng(7)
    N = 5
    qs = []
    for _ in range(N):
        a = g.standard_normal(2) + 1j * g.standard_normal(2)
        a /= np.linalg.norm(a)
        qs.append((a[0], a[1]))
    psi = inputs.product_state(qs)
    bl = [_bloch(*q) for q in qs]
    c_bf = oracle.all_expectations_bruteforce(psi)
    for x in range(1 << N):
        c_fw = oracle.family_spectrum(psi, x)
        for z in range(1 << N):
            want = np.prod([bl[j][((x >> j) & 1, (z >> j) & 1)] for j in range(N)])
            assert abs(c_bf[x, z] - want) < 2e-6
            assert abs(c_fw[z] - want) < 2e-6


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_fwht_route_equals_bruteforce(N):
    psi = inputs.haar_state(N, 11 + N)
    c_bf = oracle.all_expectations_bruteforce(psi)
    for x in range(1 << N):
        c, im = oracle.family_spectrum(psi, x, return_imag=True)
        assert np.max(np.abs(c - c_bf[x])) < 1e-12
        assert im < 1e-12


def test_bell_state_stabilizers():
    """(|00> + |11>)/sqrt2 is stabilised by XX, -YY, ZZ and II."""
    psi = np.zeros(4, dtype=np.complex64)
    psi[0] = psi[3] = 1 / np.sqrt(2)
    want = {(0, 0): 1, (0b11, 0): 1, (0, 0b11): 1, (0b11, 0b11): -1}
    c = oracle.all_expectations_bruteforce(psi)
    for x in range(4):
        for z in range(4):
            assert abs(c[x, z] - want.get((x, z), 0.0)) < 1e-7


def test_parseval_identity_and_imag():
    for N in (3, 6, 8):
        psi = inputs.unnormalised_gaussian_state(N, N)
        tot = 0.0
        for x in range(1 << N):
            c, im = oracle.family_spectrum(psi, x, return_imag=True)
            tot += np.sum(c * c)
            assert im < 1e-12
            if x == 0:
                assert abs(c[0] - 1.0) < 1e-12
        assert abs(tot / (1 << N) - 1.0) < 1e-12   # sum_P c^2/d = 1


# ------------------------------------------------------------- SRE pins
@pytest.mark.parametrize("case", [c for c in GOLDEN["t_product_state"] if c["N"] <= 7])
def test_t_product_state(case):
    psi = inputs.t_product_state(case["N"], case["k"])
    r = oracle.sre_exact(psi)
    assert abs(r["M"][0] - case["M1"]) < 1e-6
    assert abs(r["M"][1] - case["M2"]) < 1e-6
    assert abs(r["M"][2] - case["M3"]) < 1e-6
    assert r["nullity"] == case["nullity"]


@pytest.mark.parametrize("case", GOLDEN["psi_m_family_m2"])
def test_psi_m_family_moments(case):
    """SM Eqs. S4-S6 for |T>^{N/2}|0>^{N/2}."""
    N = case["N"]
    psi = inputs.t_product_state(N, N // 2)
    fam = oracle.sre_exact(psi, per_family=True)["family"]
    d = 1 << N
    m2 = fam[:, 1] / d**2
    assert np.allclose(m2, case["m2_x"], rtol=1e-6, atol=1e-15)
    assert abs(m2.mean() / case["E_x"] - 1) < 1e-6
    r2 = m2[1:].std() / m2.mean()
    assert abs(r2 / case["r2"] - 1) < 1e-6


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_exact_equals_bruteforce_sums(N):
    psi = inputs.haar_state(N, 100 + N)
    a = oracle.sre_exact(psi)
    b = oracle.sre_bruteforce(psi)
    assert np.allclose(a["M"], b["M"], atol=1e-12)
    assert np.allclose(a["S"], b["S"], rtol=1e-12)


@pytest.mark.parametrize("N,seed", [(2, 1), (3, 2), (5, 3), (6, 4), (7, 5)])
def test_stabilizer_states(N, seed):
    gates = inputs.random_clifford_gates(N, 12 * N, seed)
    psi = oracle.circuit_state(N, gates)
    r = oracle.sre_exact(psi)
    assert np.max(np.abs(r["M"])) < 1e-6
    assert r["stab_count"] == 1 << N
    assert r["nullity"] == 0


def test_ghz_state():
    N = 6
    psi = np.zeros(1 << N, dtype=np.complex64)
    psi[0] = psi[-1] = 1 / np.sqrt(2)
    r = oracle.sre_exact(psi)
    assert r["nullity"] == 0 and np.max(np.abs(r["M"])) < 1e-6


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_clifford_invariance(seed):
    N = 6
    base = inputs.random_clifford_tdoped_gates(N, 30, 5, seed)
    psi = oracle.circuit_state(N, base)
    C = inputs.random_clifford_gates(N, 40, 1000 + seed)
    psi2 = oracle.circuit_state(N, np.concatenate([base, C]))
    a, b = oracle.sre_exact(psi), oracle.sre_exact(psi2)
    assert np.allclose(a["M"], b["M"], atol=2e-6)
    assert a["nullity"] == b["nullity"]
    assert a["nullity"] <= int(np.sum(base[:, 0] == inputs.GATE_T))


def test_renyi_monotone():
    for seed in range(5):
        N = 6
        psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 40, 4, seed))
        M = oracle.sre_exact(psi)["M"]
        assert M[0] >= M[1] - 1e-9 >= -1e-6 and M[1] >= M[2] - 1e-9 and M[2] >= -1e-6


@pytest.mark.parametrize("N", [4, 6])
def test_haar_average(N):
    """E[(1/d) sum_P c^4] = 4/(d+3) over Haar states (SM, long-time limit)."""
    d = 1 << N
    vals = []
    for seed in range(200):
        S2 = oracle.sre_exact(inputs.haar_state(N, 5000 + seed))["S"][1]   # sum c^4/d^2
        vals.append(S2 * d)                                                  # (1/d) sum c^4
    vals = np.array(vals)
    want = [h for h in GOLDEN["haar"] if h["N"] == N][0]["E_sum_c4_over_d"]
    se = vals.std() / np.sqrt(len(vals))
    assert abs(vals.mean() - want) < 4 * se


def test_sm_normalisation_reading():
    """Under pi(P) = c^2/d, E_pi[c^2] = (1/d) sum c^4 = d S_2; the reading
    M_2 = -log2 E_pi[c^2] (no "- N") gives 0 for a stabilizer state and
    k log2(4/3) for |T>^k, matching Eq. SRE-def."""
    N, k = 5, 3
    for psi, want in [(oracle.circuit_state(N, inputs.random_clifford_gates(N, 40, 9)), 0.0),
                      (inputs.t_product_state(N, k), k * math.log2(4 / 3))]:
        S2 = oracle.sre_exact(psi)["S"][1]
        assert abs(-math.log2(S2 * (1 << N)) - want) < 1e-6


# ----------------------------------------------------------------- gates
def _dense(op, q0, q1, N):
    I2 = np.eye(2)
    one = {inputs.GATE_H: np.array([[1, 1], [1, -1]]) / np.sqrt(2),
           inputs.GATE_S: np.diag([1, 1j]), inputs.GATE_SDG: np.diag([1, -1j]),
           inputs.GATE_T: np.diag([1, np.exp(1j * np.pi / 4)]),
           inputs.GATE_TDG: np.diag([1, np.exp(-1j * np.pi / 4)])}
    if op != inputs.GATE_CNOT:
        U = np.array([[1.0]])
        for j in reversed(range(N)):          # qubit N-1 is the most significant factor
            U = np.kron(U, one[op] if j == q0 else I2)
        return U
    d = 1 << N
    U = np.zeros((d, d))
    for b in range(d):
        U[b ^ (1 << q1) if (b >> q0) & 1 else b, b] = 1
    return U


def test_gates_match_dense_matrices():
    N = 4
    g = np.random.default_rng(3)
    rows = []
    for _ in range(60):
        op = int(g.integers(0, 6))
        q0 = int(g.integers(0, N))
        q1 = int((q0 + 1 + g.integers(0, N - 1)) % N) if op == inputs.GATE_CNOT else 0
        rows.append((op, q0, q1))
    gates = np.array(rows, dtype=np.uint8)
    psi = inputs.haar_state(N, 3).astype(np.complex128)
    want = psi.copy()
    for op, q0, q1 in rows:
        want = _dense(op, q0, q1, N) @ want
    got = oracle.apply_gates(psi, gates)
    assert np.max(np.abs(got - want)) < 1e-12


def test_bad_gate_rejected():
    with pytest.raises(ValueError):
        oracle.apply_gates(np.ones(4, np.complex64), np.array([[inputs.GATE_CNOT, 1, 1]]))
    with pytest.raises(ValueError):
        oracle.apply_gates(np.ones(4, np.complex64), np.array([[9, 0, 0]]))


@pytest.mark.parametrize("N,seed", [(2, 1), (3, 2), (4, 3)])
def test_clifford_conjugation_matches_bruteforce(N, seed):
    """c_P(C psi) = sign * c_{P'}(psi) with C^dag P C = sign P' (Clifford
    invariance, main text); every gate type including S^dag."""
    g = np.random.default_rng(seed)
    rows = []
    for _ in range(30):
        op = int(g.choice([inputs.GATE_H, inputs.GATE_S, inputs.GATE_SDG, inputs.GATE_CNOT])) if N > 1 \
            else int(g.choice([inputs.GATE_H, inputs.GATE_S, inputs.GATE_SDG]))
        q0 = int(g.integers(0, N))
        q1 = int((q0 + 1 + g.integers(0, N - 1)) % N) if op == inputs.GATE_CNOT else 0
        rows.append((op, q0, q1))
    C = np.array(rows, dtype=np.uint8)
    psi = inputs.haar_state(N, seed)
    Cpsi = oracle.apply_gates(psi, C).astype(np.complex64)
    for x in range(1 << N):
        for z in range(1 << N):
            x2, z2, sg = oracle.clifford_conjugate(N, C, x, z)
            assert abs(oracle.pauli_expectation(Cpsi, x, z) - sg * oracle.pauli_expectation(psi, x2, z2)) < 1e-5


def test_clifford_conjugation_rejects_t():
    with pytest.raises(ValueError):
        oracle.clifford_conjugate(2, np.array([[inputs.GATE_T, 0, 0]], dtype=np.uint8), 1, 0)


# -------------------------------------------------------------- marginal
@pytest.mark.parametrize("N", [1, 3, 6, 9])
def test_marginal_routes(N):
    psi = inputs.unnormalised_gaussian_state(N, 40 + N)
    p1 = oracle.x_marginal(psi, "direct")
    p2 = oracle.x_marginal(psi, "wht")
    assert np.max(np.abs(p1 - p2)) < 1e-14
    assert abs(p2.sum() - 1.0) < 1e-12
    for x in (0, 1, (1 << N) - 1):
        assert abs(oracle.x_marginal_one(psi, x) - p1[x]) < 1e-15
    if N <= 6:
        for x in range(1 << N):
            c = oracle.family_spectrum(psi, x)
            assert abs(np.sum(c * c) / (1 << N) - p2[x]) < 1e-13


def test_fwht_real_is_hadamard_matrix():
    n = 5
    H = np.array([[1.0]])
    for _ in range(n):
        H = np.block([[H, H], [H, -H]])
    v = np.random.default_rng(1).standard_normal(1 << n)
    assert np.allclose(oracle.fwht_real(v), H @ v, atol=1e-12)


# -------------------------------------------------------------- sampling
def test_inverse_cdf_definition():
    w = [0.0, 1.0, 0.0, 2.0, 1.0]   # C = 0,1,1,3,4; total 4
    assert oracle.inverse_cdf(w, 0.0) == 1
    assert oracle.inverse_cdf(w, 0.2499) == 1
    assert oracle.inverse_cdf(w, 0.25) == 3
    assert oracle.inverse_cdf(w, 0.7499) == 3
    assert oracle.inverse_cdf(w, 0.75) == 4
    assert oracle.inverse_cdf(w, 1.0 - 2**-53) == 4
    assert oracle.inverse_cdf([0.0, 0.0, 5.0, 0.0], 0.999) == 2


def test_mc_marginal_draw_frequencies():
    """Families 1.. draw x ~ p(x | x != 0)."""
    N = 3
    psi = inputs.haar_state(N, 77)
    p = oracle.x_marginal(psi)
    r = oracle.mc_marginal(psi, 4001, 1, seed=5)
    assert r["xs"][0] == 0
    counts = np.bincount(r["xs"][1:].astype(np.int64), minlength=1 << N)
    q = p.copy()
    q[0] = 0
    q /= q.sum()
    assert counts[0] == 0
    chi2 = np.sum((counts[1:] - 4000 * q[1:]) ** 2 / (4000 * q[1:]))
    assert chi2 < 28   # 6 dof; P(chi2 > 28) ~ 1e-4


def test_mc_marginal_pairs_are_inverse_cdf_draws():
    N = 5
    psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 30, 3, 4))
    r = oracle.mc_marginal(psi, 6, 4, seed=9, ctr0=17)
    p = oracle.x_marginal(psi)
    p[0] = 0.0
    for i in range(6):
        x = int(r["xs"][i])
        assert x == (0 if i == 0 else oracle.inverse_cdf(p, oracle.mc_draw(9, 17, i, 0)))
        c = oracle.family_spectrum(psi, x)
        for k in range(4):
            z = int(r["zs"][i, k])
            assert z == oracle.inverse_cdf(c * c, oracle.mc_draw(9, 17, i, 1 + k))
            assert abs(r["c"][i, k] - oracle.pauli_expectation(psi, x, z)) < 1e-12


def test_mc_marginal_stabilizer_is_exactly_zero():
    N = 6
    psi = oracle.circuit_state(N, inputs.random_clifford_gates(N, 60, 3))
    r = oracle.mc_marginal(psi, 20, 8, seed=1)
    assert np.max(np.abs(r["M"])) < 1e-6 and np.max(np.abs(r["M_rb"])) < 1e-6
    assert np.allclose(np.abs(r["c"]), 1.0, atol=1e-6)


def test_mc_marginal_unbiased():
    """E over seeds of mean c^2 = E_pi[c^2] = (1/d) sum c^4."""
    N = 5
    psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 40, 4, 8))
    want = oracle.sre_exact(psi)["S"][1] * (1 << N)
    est = [2.0 ** (-oracle.mc_marginal(psi, 8, 4, seed=s)["M"][1]) for s in range(300)]
    est_rb = [2.0 ** (-oracle.mc_marginal(psi, 8, 1, seed=s)["M_rb"][1]) for s in range(300)]
    for e in (np.array(est), np.array(est_rb)):
        assert abs(e.mean() - want) < 4 * e.std() / np.sqrt(len(e)) + 1e-12


def test_mc_marginal_haar_needs_the_x0_stratum():
    """For a Haar state the identity alone holds about a quarter of
    sum_P c^4 while p(0) ~ 2/d: with x = 0 as its own stratum the estimate of
    M_2 sits on the closed form log2(d+3) - 2 (SM Sec. I reasoning)."""
    N = 14
    psi = inputs.haar_state(N, 14)
    r = oracle.mc_marginal(psi, 120, 4, seed=7)
    m2 = math.log2((1 << N) + 3) - 2
    assert abs(r["M_rb"][1] - m2) < 4 * r["err_rb"][1] + 0.01
    assert abs(r["M"][1] - m2) < 4 * r["err"][1] + 0.02
    # what the stratum adds: the x = 0 family's share of sum c^4
    c0 = oracle.family_spectrum(psi, 0)
    share = np.sum(c0**4) / (4.0 * (1 << N) / ((1 << N) + 3))   # sum_P c^4 = 4d/(d+3)
    assert 0.2 < share < 0.3


def test_mc_uniform_unbiased():
    """SM Sec. I: S_hat is unbiased for S = sum_x m_{2;x}."""
    N = 6
    psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 40, 3, 2))
    d = 1 << N
    S = oracle.sre_exact(psi)["S"][1]
    est = np.array([2.0 ** (-(oracle.mc_uniform(psi, 12, seed=s)["M"][1] + N)) for s in range(300)])
    assert abs(est.mean() - S) < 4 * est.std() / np.sqrt(len(est))
    r = oracle.mc_uniform(psi, 12, seed=3)
    assert r["xs"][0] == 0 and np.all(r["xs"][1:] >= 1) and np.all(r["xs"][1:] < d)


def test_mc_all_families_is_exact_at_large_sample():
    """With x = 0 forced and every other x drawn uniformly many times the
    uniform estimator converges to the exact S."""
    N = 4
    psi = inputs.haar_state(N, 3)
    ex = oracle.sre_exact(psi)["M"]
    mc = oracle.mc_uniform(psi, 20000, seed=1)
    assert np.all(np.abs(mc["M"] - ex) < 5 * mc["err"] + 1e-9)


# ------------------------------------------- MC standard errors (Eq. stdM)
# The error bars of both MC estimators are pinned against the spread of the
# estimates themselves over many seeds, which no formula in the oracle enters.
#
# alpha = 1 is exact at any sample size: M_1 is linear in the per-family
# values (uniform: M_1 = m_0 + (d-1) mean h_x - N; marginal: M_1 = p(0) G_0 +
# (1 - p(0)) mean g_x), and the oracle's error bar is the population standard
# deviation of the nm drawn families over sqrt(nm) (times (d-1), resp.
# (1 - p(0))), so E[err^2] = ((nm-1)/nm) Var(M_1) exactly. At nm = 2 that
# separates sqrt(nm) from sqrt(nm+1) (a factor 2/3 in the variance) and, on a
# state with p(0) = 1/4, a dropped (1 - p(0)) (a factor 16/9).
#
# alpha = 2, 3 use the delta method (Eq. stdM: 1/(|1-alpha| ln 2 sqrt(N_x))
# times the relative spread), valid once the relative error of S is small:
# checked at 400-800 families, where the mean error bar must match the
# standard deviation of M_hat within 15% (500 seeds: about 3% sampling noise
# on that standard deviation); a dropped ln 2 is off by 1/ln 2 = 1.44.
def _sigma_states():
    N = 8
    mixed = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 80, 4, 11))   # p(0) ~ 0.01
    local = inputs.t_product_state(N, 2)                                                 # p(0) = 1/4
    return mixed, local


def _spread(psi, mode, n_x, seeds, zpx=4):
    """(estimates, error bars) over seeds, per estimator: {name: (M[K,3], err[K,3])}."""
    acc = {}
    for s in seeds:
        if mode == "uniform":
            r = oracle.mc_uniform(psi, n_x, seed=s)
            acc.setdefault("uniform", ([], []))
            acc["uniform"][0].append(r["M"]); acc["uniform"][1].append(r["err"])
        else:
            r = oracle.mc_marginal(psi, n_x, zpx, seed=s)
            for nm_, mk, ek in (("z-sample", "M", "err"), ("per-family", "M_rb", "err_rb")):
                acc.setdefault(nm_, ([], []))
                acc[nm_][0].append(r[mk]); acc[nm_][1].append(r[ek])
    return {k: (np.array(v[0]), np.array(v[1])) for k, v in acc.items()}


def _sigma_small_n_ratios():
    """Var-ratio E[err_1^2] nm/(nm-1) / Var(M_1) at n_x = 3 (nm = 2 drawn
    families), 6000 seeds, for every estimator and both states."""
    out = {}
    mixed, local = _sigma_states()
    nm = 2
    for sname, psi in (("mixed", mixed), ("local", local)):
        for mode in ("uniform", "marginal"):
            for est, (M, e) in _spread(psi, mode, nm + 1, range(5000, 11000), zpx=2).items():
                out[(sname, est)] = np.mean(e[:, 0] ** 2) * nm / (nm - 1) / np.var(M[:, 0], ddof=1)
    return out


def _sigma_large_n_ratios():
    """mean err / std M for alpha = 1, 2, 3 at 800 (uniform) and 400
    (marginal) families, 500 seeds, on the mixed-support state."""
    mixed, _ = _sigma_states()
    out = {}
    for mode, n_x in (("uniform", 800), ("marginal", 400)):
        for est, (M, e) in _spread(mixed, mode, n_x, range(2000, 2500)).items():
            out[est] = e.mean(axis=0) / M.std(axis=0, ddof=1)
    return out


def _sigma_pins_pass():
    small = _sigma_small_n_ratios()
    if any(abs(v - 1.0) > 0.12 for v in small.values()):
        return False
    large = _sigma_large_n_ratios()
    return all(abs(r - 1.0) < 0.15 for v in large.values() for r in v)


def test_mc_standard_error_exact_at_small_n():
    for key, v in _sigma_small_n_ratios().items():
        assert abs(v - 1.0) < 0.12, (key, v)


def test_mc_standard_error_matches_spread():
    for est, v in _sigma_large_n_ratios().items():
        for a in range(3):
            assert abs(v[a] - 1.0) < 0.15, (est, a + 1, v[a])


@pytest.mark.parametrize("m", [5, 6, 7])
def test_sigma_mutations(m):
    """5: ln 2 dropped; 6: (1 - p(0)) dropped; 7: sqrt(n) -> sqrt(n + 1).
    Each must fail the standard-error pins."""
    oracle.set_mutation(m)
    try:
        assert not _sigma_pins_pass()
    finally:
        oracle.set_mutation(0)


# ------------------------------------------------------------- mutations
def _pins_pass():
    """A compact subset of the pins above; False if any fails."""
    try:
        for name in ("T", "+i"):
            psi = np.array(ONE_QUBIT[name], dtype=np.complex64)
            for (x, z), want in EXPECTED_ONE_QUBIT[name].items():
                if abs(oracle.pauli_expectation(psi, x, z) - want) > 1e-7:
                    return False
                if abs(oracle.family_spectrum(psi, x)[z] - want) > 1e-7:
                    return False
        psi = np.zeros(4, dtype=np.complex64)
        psi[0] = psi[3] = 1 / np.sqrt(2)
        c = oracle.family_spectrum(psi, 3)
        if abs(c[3] + 1) > 1e-7 or abs(c[0] - 1) > 1e-7:
            return False
        g = np.random.default_rng(5)
        a = g.standard_normal(4) + 1j * g.standard_normal(4)
        psi = inputs.product_state([(a[0], a[1]), (a[2], a[3])])
        bl = [_bloch(a[0], a[1]), _bloch(a[2], a[3])]
        for x in range(4):
            cf = oracle.family_spectrum(psi, x)
            for z in range(4):
                want = bl[0][(x & 1, z & 1)] * bl[1][(x >> 1, z >> 1)]
                if abs(cf[z] - want) > 2e-6 or abs(oracle.pauli_expectation(psi, x, z) - want) > 2e-6:
                    return False
        r = oracle.sre_exact(inputs.t_product_state(4, 2))
        if abs(r["M"][1] - 2 * math.log2(4 / 3)) > 1e-6:
            return False
        return True
    finally:
        pass


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_mutations(m):
    """1: phase i^{x.z} dropped; 2: conjugation order swapped; 3: wrong
    output index; 4: "- N" dropped from M_2. Each must fail a pin."""
    assert _pins_pass()
    oracle.set_mutation(m)
    try:
        assert not _pins_pass()
    finally:
        oracle.set_mutation(0)
    assert _pins_pass()


# ------------------------------------------------ fluctuation ratio r_2
def _r2_psi_m_closed_form(N):
    """SM, analytic fluctuation ratio (Eq. sm-psi-m-ratio-exact) for
    |T>^{N/2} (x) |0>^{N/2}, even N."""
    h = N // 2
    a = (5 / 4) ** h - 1
    b = 4 ** h - 1
    c = (3 / 2) ** h - 1
    return (8 / 3) ** h * math.sqrt(a / b - c * c / (b * b))


@pytest.mark.parametrize("N", [2, 4, 6, 8, 10])
def test_r2_product_magic_state_closed_form(N):
    psi = inputs.t_product_state(N, N // 2)
    assert abs(oracle.fluctuation_ratio(psi) - _r2_psi_m_closed_form(N)) < 1e-9 * _r2_psi_m_closed_form(N)


def test_r2_closed_form_large_n_asymptote():
    # the closed form's leading term grows as (20/9)^{N/4} (SM, Eq. sm-psi-m-ratio-asym)
    r40, r44 = _r2_psi_m_closed_form(40), _r2_psi_m_closed_form(44)
    assert abs(r44 / r40 - (20 / 9)) < 1e-2


@pytest.mark.parametrize("N", [4, 6, 8])
def test_r2_family_values_product_magic_state(N):
    """SM Eq. sm-psi-m-m2x: m_{2;x} = 4^{-N} sum_z c^4 = 2^{-3N/2-k} when x has
    weight k on the |T> qubits and none on the |0> qubits, else 0."""
    h = N // 2
    fam = oracle.sre_exact(inputs.t_product_state(N, h), per_family=True)["family"]
    for x in range(1 << N):
        m = fam[x, 1] / 4.0 ** N
        if x >> h:
            assert m < 1e-15
        else:
            assert abs(m - 2.0 ** (-1.5 * N - bin(x).count("1"))) < 1e-12 * 2.0 ** (-1.5 * N)


def test_r2_stabilizer_state_is_zero():
    # |0>^N: only the x = 0 family is nonzero, so every x != 0 has m_x = 0
    assert oracle.fluctuation_ratio(inputs.basis_state(6, 0)) == 0.0


# ------------------------------------------------- two-qubit gates (brick walls)
_PAULI1 = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1, -1])]


def test_two_qubit_clifford_table_is_the_group():
    """11520 = |C_2| modulo phase; every element unitary and mapping Pauli
    operators to signed Pauli operators; closed under products."""
    t = inputs.two_qubit_clifford_table()
    assert t.shape == (11520, 4, 4)
    paulis = [np.kron(a, b) for a in _PAULI1 for b in _PAULI1]
    g = np.random.default_rng(3)
    for u in t[g.integers(0, len(t), 64)]:
        assert np.allclose(u.conj().T @ u, np.eye(4), atol=1e-12)
        for p in paulis[1:]:
            q = u @ p @ u.conj().T
            assert any(np.allclose(q, s * r, atol=1e-9) for r in paulis for s in (1, -1))
    keys = {inputs._key(u) for u in t}
    for _ in range(64):
        a, b = t[g.integers(0, len(t))], t[g.integers(0, len(t))]
        assert inputs._key(a @ b) in keys


def _dense_two_qubit(N, u, q0, q1):
    """The 2^N x 2^N matrix of u on (q0, q1), built from index arithmetic."""
    d = 1 << N
    full = np.zeros((d, d), dtype=np.complex128)
    for b in range(d):
        lin = ((b >> q0) & 1) + 2 * ((b >> q1) & 1)
        rest = b & ~((1 << q0) | (1 << q1))
        for lo in range(4):
            bo = rest | ((lo & 1) << q0) | ((lo >> 1) << q1)
            full[bo, b] += u[lo, lin]
    return full


@pytest.mark.parametrize("pair", [(0, 1), (2, 0), (1, 3), (3, 2)])
def test_two_qubit_gate_vs_dense(pair):
    N = 4
    g = np.random.default_rng(sum(pair))
    psi = g.standard_normal(16) + 1j * g.standard_normal(16)
    u = inputs.haar_two_qubit(g)
    out = oracle.apply_two_qubit(psi, u[None], [pair])
    assert np.allclose(out, _dense_two_qubit(N, u, *pair) @ psi, atol=1e-12)


def test_two_qubit_gate_kron_of_one_qubit_gates():
    # kron(B, A) on (q0, q1) is A on q0 and B on q1 (local index bit(q0) + 2 bit(q1))
    g = np.random.default_rng(9)
    psi = g.standard_normal(8) + 1j * g.standard_normal(8)
    a = inputs.haar_two_qubit(g)[:2, :2]
    a = np.linalg.qr(a)[0]
    out = oracle.apply_two_qubit(psi, np.kron(np.eye(2), a)[None], [(2, 0)])
    ref = np.einsum("ij,jab->iab", a, psi.reshape(2, 2, 2)).reshape(-1)   # axis 0 of the C-order reshape is qubit 2
    assert np.allclose(out, ref, atol=1e-12)


def test_brickwall_clifford_preserves_sre_and_haar_norm():
    N = 6
    psi = inputs.t_product_state(N, 3).astype(np.complex128)
    m, p = inputs.brickwall_circuit(N, 2 * N, "clifford", 5)
    after = oracle.apply_two_qubit(psi, m, p)
    a, b = oracle.sre_exact(psi.astype(np.complex64)), oracle.sre_exact(after.astype(np.complex64))
    assert np.allclose(a["M"], b["M"], atol=1e-6)
    assert abs(b["M"][1] - 3 * math.log2(4 / 3)) < 1e-6
    zero = oracle.apply_two_qubit(inputs.basis_state(N, 0), m, p)
    assert oracle.sre_exact(zero.astype(np.complex64))["nullity"] == 0
    mh, ph = inputs.brickwall_circuit(N, 5, "haar", 6)
    out = oracle.apply_two_qubit(inputs.haar_state(N, 2), mh, ph)
    assert abs(np.vdot(out, out).real - 1.0) < 1e-6


# ---------------------------------------------------- mixed-state SRE (SM)
@pytest.mark.parametrize("N,NA", [(3, 1), (4, 2), (5, 3), (6, 5), (5, 5), (7, 2)])
def test_mixed_route_equals_definition(N, NA):
    psi = inputs.unnormalised_gaussian_state(N, 70 + N + NA)
    a = oracle.sre_mixed(psi, NA, "partial")
    b = oracle.sre_mixed(psi, NA, "bruteforce")
    assert np.allclose(a["W"], b["W"], rtol=1e-12, atol=1e-14)
    assert abs(a["S2"] - b["S2"]) < 1e-12


@pytest.mark.parametrize("N", [3, 6, 8])
def test_mixed_full_subsystem_is_the_pure_sre(N):
    psi = inputs.haar_state(N, 80 + N)
    m = oracle.sre_mixed(psi, N)
    p = oracle.sre_exact(psi)
    assert abs(m["S2"]) < 1e-12
    assert np.allclose(m["M"], p["M"], atol=1e-10)


@pytest.mark.parametrize("NA,NB", [(1, 3), (3, 2), (4, 4)])
def test_mixed_product_state_is_pure_on_a(NA, NB):
    """|T>^{NA} (x) (Haar on B): rho_A = |T><T|^{NA}, S_2 = 0, M_2 =
    NA log2(4/3), M_3 = NA (1/2) log2(8/5) (one |T>: sum_P c^6 = 1 + 2/8)."""
    t = inputs.t_product_state(NA, NA).astype(np.complex128)
    b = inputs.haar_state(NB, 90 + NB).astype(np.complex128)
    psi = np.kron(b, t)                            # A = the low NA qubits
    m = oracle.sre_mixed(psi, NA)
    assert abs(m["S2"]) < 1e-9
    assert abs(m["M"][1] - NA * math.log2(4 / 3)) < 1e-9
    assert abs(m["M"][2] - NA * 0.5 * math.log2(8 / 5)) < 1e-9


@pytest.mark.parametrize("NA", [1, 2, 4])
def test_mixed_bell_pairs_maximally_mixed(NA):
    """Qubit i of A in |Phi+> with qubit NA + i of B: rho_A = I / d_A, so only
    the identity has c != 0: S_2 = N_A, and Eq. Msre-mixed (which subtracts
    S_2 for every alpha) gives M_alpha = N_A (2 - alpha)/(alpha - 1): M_2 = 0,
    M_3 = -N_A / 2."""
    N = 2 * NA
    psi = np.zeros(1 << N, dtype=np.complex128)
    for a in range(1 << NA):
        psi[a | (a << NA)] = 1.0
    psi /= np.linalg.norm(psi)
    m = oracle.sre_mixed(psi, NA)
    assert abs(m["S2"] - NA) < 1e-12
    assert abs(m["M"][1]) < 1e-12 and abs(m["M"][2] + NA / 2) < 1e-12
    assert np.allclose(m["W"][:3], 1.0) and math.isnan(m["M"][0])


def test_mixed_ghz_two_component_mixture():
    """GHZ on 6 qubits, A = 3 qubits: rho_A = (|000><000| + |111><111|)/2;
    the even-weight Z strings have c = 1, all else 0: S_2 = 1, M_2 = 0 and
    M_3 = -log2(4 / 8^3) / 2 - 3 - 1 = -1/2."""
    psi = np.zeros(64, dtype=np.complex128)
    psi[0] = psi[63] = 1 / math.sqrt(2)
    m = oracle.sre_mixed(psi, 3)
    assert abs(m["S2"] - 1.0) < 1e-12 and abs(m["M"][1]) < 1e-12 and abs(m["M"][2] + 0.5) < 1e-12
    assert np.allclose(m["W"][:3], 4.0)
