"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (FP32 SIMT path): |dc| <= 1e-6 per Pauli expectation, |dM_a| <=
1e-5 (base-2 units); nullity, stabilizer counts, sampled x and z indices and
Philox words bit-exact; FP64 paths (nullity recheck arithmetic, x-marginal)
1e-12."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_00761_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_C = 1e-6
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


def sample_xs(N, k, seed):
    d = 1 << N
    g = np.random.default_rng(seed)
    xs = {0, 1, d - 1, 1 << (N - 1), (1 << (N - 1)) | 1, d // 3}
    xs |= set(int(v) for v in g.integers(0, d, size=k))
    return sorted(x for x in xs if 0 <= x < d)


def draw_within_bound(zg, zo, w_oracle, w_gpu, u, range_log2=13):
    """A z drawn from FP32-computed weights against the oracle's FP64 draw:
    equal, or both on the same side of the target within the propagated
    bound delta = sum |w_gpu - w_oracle| (each cumulative sum and the target
    differ by at most delta) plus the sampler's fixed-point rounding inside a
    z-range (half a quantum of 2^-31 range weight per entry, 2^RL entries).
    Returns (valid, exact)."""
    if zg == zo:
        return True, True
    delta = float(np.sum(np.abs(w_gpu - w_oracle))) + 1e-12
    wr = max(float(np.sum(w_oracle[(zz >> range_log2) << range_log2:((zz >> range_log2) + 1) << range_log2]))
             for zz in (zg, zo))
    delta += 2.0 ** (range_log2 - 32) * wr
    C = np.cumsum(w_oracle)
    t = u * C[-1]
    lo = C[zg - 1] if zg > 0 else 0.0
    return bool(C[zg] > t - 2 * delta and lo <= t + 2 * delta), False


# ------------------------------------------------------------------ RNG
def test_philox_device_matches_oracle(sre):
    g = np.random.default_rng(1)
    rows = g.integers(0, 2**63, size=(64, 6), dtype=np.int64)
    rows[0] = 0
    rows[1] = -1                                   # all ones
    out = sre.sre_philox_blocks(torch.from_numpy(rows).cuda()).cpu().numpy().view(np.uint64)
    for i in range(rows.shape[0]):
        r = rows[i].view(np.uint64)
        assert np.array_equal(out[i], oracle.philox4x64_10(r[:4], r[4:]))


def test_norm2(sre):
    for N in (1, 5, 12, 20):
        psi = inputs.unnormalised_gaussian_state(N, N)
        assert abs(sre.sre_norm2(dev(psi)) / oracle.norm2(psi) - 1) < 1e-12


# ------------------------------------------------------------- spectra
@pytest.mark.parametrize("N", list(range(1, 9)))
def test_family_spectrum_all_x(sre, N):
    psi = inputs.unnormalised_gaussian_state(N, 50 + N)
    p = dev(psi)
    for x in range(1 << N):
        c = sre.sre_family_spectrum(p, x).cpu().numpy()
        assert np.max(np.abs(c - oracle.family_spectrum(psi, x))) < TOL_C, x


@pytest.mark.parametrize("N", [9, 10, 11, 12, 13, 14, 15])
def test_family_spectrum_single_pass(sre, N):
    psi = inputs.haar_state(N, 60 + N)
    p = dev(psi)
    for x in sample_xs(N, 6, N):
        c = sre.sre_family_spectrum(p, x).cpu().numpy()
        assert np.max(np.abs(c - oracle.family_spectrum(psi, x))) < TOL_C, x


@pytest.mark.parametrize("N,kw", [(16, {}), (17, {}), (18, {}), (18, {"radix_log2": 10, "tile_log2": 4}),
                                  (19, {"radix_log2": 11}), (20, {}), (22, {"tile_log2": 5})])
def test_family_spectrum_multi_pass(sre, N, kw):
    psi = inputs.haar_state(N, 70 + N)
    p = dev(psi)
    for x in sample_xs(N, 3, N):
        c = sre.sre_family_spectrum(p, x, **kw).cpu().numpy()
        assert np.max(np.abs(c - oracle.family_spectrum(psi, x))) < TOL_C, (x, kw)


def test_family_spectrum_n24_full_size(sre):
    """Headline size: 2 passes (10 + 13 bits), sampled families."""
    N = 24
    psi = inputs.haar_state(N, 24)
    p = dev(psi)
    for x in (0, 0x9A3C51, (1 << 23) | 5):
        c = sre.sre_family_spectrum(p, x).cpu().numpy()
        assert np.max(np.abs(c - oracle.family_spectrum(psi, x))) < TOL_C, x


def test_family_spectrum_three_pass(sre):
    N = 25
    psi = inputs.haar_state(N, 25)
    p = dev(psi)
    for x in (0, (1 << 24) | 0x1234):
        c = sre.sre_family_spectrum(p, x).cpu().numpy()
        assert np.max(np.abs(c - oracle.family_spectrum(psi, x))) < TOL_C, x


def test_family_spectrum_product_state_large(sre):
    """Product states: c_{x,z} = prod_j c^(j), checked on sampled z at N=24."""
    N = 24
    g = np.random.default_rng(5)
    qs = []
    for _ in range(N):
        a = g.standard_normal(2) + 1j * g.standard_normal(2)
        a /= np.linalg.norm(a)
        qs.append((a[0], a[1]))
    psi = inputs.product_state(qs)
    bl = []
    for a0, a1 in qs:
        X = 2 * (np.conj(a0) * a1).real
        Y = 2 * (np.conj(a0) * a1).imag
        Z = abs(a0) ** 2 - abs(a1) ** 2
        bl.append({(0, 0): 1.0, (0, 1): Z, (1, 0): X, (1, 1): Y})
    p = dev(psi)
    for x in (0, 0xABCDE1, (1 << 24) - 1):
        c = sre.sre_family_spectrum(p, x).cpu().numpy()
        for z in g.integers(0, 1 << N, size=200):
            want = np.prod([bl[j][((x >> j) & 1, (int(z) >> j) & 1)] for j in range(N)])
            assert abs(c[z] - want) < TOL_C + 1e-6   # complex64 input rounding


@pytest.mark.parametrize("N", [1, 3, 8, 12, 13, 14, 16])
def test_family_spectrum_f64(sre, N):
    psi = inputs.haar_state(N, 80 + N)
    p = dev(psi)
    for x in sample_xs(N, 3, N):
        c = sre.sre_family_spectrum_f64(p, x).cpu().numpy()
        assert np.max(np.abs(c - oracle.family_spectrum(psi, x))) < 1e-12, x


# ---------------------------------------------------------------- exact
def _check_exact(r, ref, N):
    assert np.max(np.abs(np.array(r["M"]) - ref["M"])) < TOL_M, (r["M"], ref["M"])
    assert r["stab_count"] == ref["stab_count"]
    assert r["nullity"] == ref["nullity"]
    assert abs(r["parseval"] - 1.0) < 1e-5


def test_exact_n10_workload(sre):
    w = inputs.workload_n10_states()
    states = [w["haar"], oracle.circuit_state(10, w["tdoped_gates"]), w["t4"]]
    for psi in states:
        ref = oracle.sre_exact(psi)
        r = sre.sre_exact(dev(psi), allow_nullity_error=True)
        _check_exact(r, ref, 10)
    r = sre.sre_exact(dev(w["t4"]))
    assert abs(r["M"][1] - 4 * math.log2(4 / 3)) < TOL_M and r["nullity"] == 4


@pytest.mark.parametrize("N", [2, 4, 6, 8, 11, 12, 13])
def test_exact_vs_oracle(sre, N):
    gates = inputs.random_clifford_tdoped_gates(N, 6 * N, 3, 300 + N)
    psi = oracle.circuit_state(N, gates)
    _check_exact(sre.sre_exact(dev(psi), allow_nullity_error=True), oracle.sre_exact(psi), N)
    h = inputs.haar_state(N, 400 + N)
    _check_exact(sre.sre_exact(dev(h), allow_nullity_error=True), oracle.sre_exact(h), N)


@pytest.mark.parametrize("N,k", [(1, 1), (2, 0), (5, 3), (9, 9), (14, 7), (15, 5), (16, 8), (17, 3), (18, 9),
                                 (20, 6)])
def test_exact_t_product_closed_form(sre, N, k):
    r = sre.sre_exact(dev(inputs.t_product_state(N, k)))
    assert abs(r["M"][0] - k / 2) < TOL_M
    assert abs(r["M"][1] - k * math.log2(4 / 3)) < TOL_M
    assert abs(r["M"][2] - (k / 2) * math.log2(8 / 5)) < TOL_M
    assert r["nullity"] == k and r["stab_count"] == 1 << (N - k)


@pytest.mark.parametrize("N", [2, 5, 9, 14, 16, 18])
def test_exact_stabilizer_states(sre, N):
    psi = oracle.circuit_state(N, inputs.random_clifford_gates(N, 8 * N, 900 + N))
    r = sre.sre_exact(dev(psi))
    assert np.max(np.abs(r["M"])) < TOL_M
    assert r["nullity"] == 0 and r["stab_count"] == 1 << N


def test_exact_n18_workload(sre):
    """N=18 T-doped circuits (eta x n_T grid, first four of twelve): sampled
    families against the oracle plus the invariants that hold at any size."""
    for spec in inputs.workload_n18_gate_lists()[:4]:
        psi = oracle.circuit_state(18, spec["gates"])
        p = dev(psi)
        r = sre.sre_exact(p)
        assert abs(r["parseval"] - 1) < 1e-5
        assert r["M"][0] >= r["M"][1] - TOL_M and r["M"][1] >= r["M"][2] - TOL_M and r["M"][2] > -TOL_M
        assert 0 <= r["nullity"] <= spec["n_t"]
        if spec["n_t"] == 0:
            assert np.max(np.abs(r["M"])) < TOL_M and r["nullity"] == 0
        for x in sample_xs(18, 2, spec["seed"]):
            c = sre.sre_family_spectrum(p, x).cpu().numpy()
            assert np.max(np.abs(c - oracle.family_spectrum(psi, x))) < TOL_C


@pytest.mark.parametrize("NA,NB", [(8, 8), (9, 8), (9, 9), (10, 10)])
def test_exact_product_additivity(sre, NA, NB):
    """N = 16..20, beyond the oracle's full sweep in test time: M_a, the
    nullity and the stabilizer count of a product state are the sums
    (product) of those of its factors, each factor's taken from the oracle."""
    a = inputs.haar_state(NA, 500 + NA)
    b = oracle.circuit_state(NB, inputs.random_clifford_tdoped_gates(NB, 6 * NB, 3, 600 + NB))
    ra, rb = oracle.sre_exact(a), oracle.sre_exact(b)
    r = sre.sre_exact(dev(np.kron(a, b)), allow_nullity_error=True)
    assert np.max(np.abs(np.array(r["M"]) - (np.array(ra["M"]) + rb["M"]))) < TOL_M, (r["M"], ra["M"], rb["M"])
    assert r["nullity"] == ra["nullity"] + rb["nullity"]
    assert r["stab_count"] == ra["stab_count"] * rb["stab_count"]


def test_exact_clifford_invariance_multipass(sre):
    N = 16
    base = inputs.random_clifford_tdoped_gates(N, 0, 4, 77, n_t=6, first_block=32)
    psi = oracle.circuit_state(N, base)
    C = inputs.random_clifford_gates(N, 64, 78)
    psi2 = oracle.circuit_state(N, np.concatenate([base, C]))
    a = sre.sre_exact(dev(psi))
    b = sre.sre_exact(dev(psi2))
    assert np.max(np.abs(np.array(a["M"]) - b["M"])) < 2 * TOL_M
    assert a["nullity"] == b["nullity"] <= 6


@pytest.mark.parametrize("N", [6, 13, 16, 18])
def test_nullity_wide_tolerance(sre, N):
    """Qubit 0 with <Y> = 1 - 5e-4, the rest |0>: the Y family's largest
    |c| is 1 - 5e-4 and it holds no exact stabilizer. At eps = 1e-3 its 2^(N-1)
    strings count (nullity 0), at eps = 1e-6 they do not (nullity 1); both
    readings of the nullity definition, with the oracle's count up to N = 8."""
    phi = math.acos(1.0 - 5e-4)
    q0 = (1 / math.sqrt(2), 1j * complex(math.cos(phi), math.sin(phi)) / math.sqrt(2))
    psi = inputs.product_state([q0] + [inputs.ZERO_QUBIT] * (N - 1))
    p = dev(psi)
    assert sre.stabilizer_nullity(p, eps=1e-3) == (0, 1 << N)
    assert sre.stabilizer_nullity(p, eps=1e-6) == (1, 1 << (N - 1))
    r = sre.sre_exact(p, eps_null=1e-3)
    assert r["nullity"] == 0 and r["stab_count"] == 1 << N
    if N <= 8:
        assert oracle.sre_exact(psi, eps=1e-3)["nullity"] == 0
        assert oracle.sre_exact(psi, eps=1e-6)["nullity"] == 1


@pytest.mark.parametrize("N", [8, 12, 16])
def test_nullity_count_not_a_subgroup(sre, N):
    """Every qubit with <Z> = 1 - 6e-4, eps = 1e-3: exactly the strings of
    Z-weight <= 1 lie within eps of 1 (1 + N of them, not a power of two, so
    the nullity is undefined); their packed z' span more than six dimensions,
    so the recount sums at each listed z'. Oracle count up to N = 8."""
    th = math.acos(1.0 - 6e-4) / 2
    psi = inputs.product_state([(math.cos(th), math.sin(th))] * N)
    r = sre.sre_exact(dev(psi), eps_null=1e-3, allow_nullity_error=True)
    assert r["stab_count"] == 1 + N and r["nullity"] == -1
    if N <= 8:
        assert oracle.sre_exact(psi, eps=1e-3)["stab_count"] == 1 + N


@pytest.mark.parametrize("k,seed", [(4, 1), (5, 2), (6, 3), (7, 4)])
def test_nullity_coset_families(sre, k, seed):
    """A random k-qubit stabilizer state next to |0>^(10-k): a family with a
    stabilizer holds 2^(10-k) of them or more, their packed z' a coset of 3 to
    6 dimensions (bin sums, in two and four chunks for 5 and 6), the x = 0
    family's beyond the list (FP64 transform). Count, nullity and M_a against
    the oracle."""
    N = 10
    top = oracle.circuit_state(k, inputs.random_clifford_gates(k, 12 * k, 950 + seed))
    low = np.zeros(1 << (N - k), dtype=np.complex128)
    low[0] = 1.0
    psi = np.kron(top, low)
    ref = oracle.sre_exact(psi)
    r = sre.sre_exact(dev(psi))
    assert r["stab_count"] == ref["stab_count"] == 1 << N and r["nullity"] == 0
    assert np.max(np.abs(np.array(r["M"]) - ref["M"])) < TOL_M


def test_nullity_entry_point(sre):
    nu, cnt = sre.stabilizer_nullity(dev(inputs.t_product_state(12, 5)))
    assert nu == 5 and cnt == 1 << 7


def test_zero_state_rejected(sre):
    with pytest.raises(sre.SreError) as e:
        sre.sre_exact(torch.zeros(1 << 6, dtype=torch.complex64, device="cuda"))
    assert e.value.status == sre.SRE_EZERO


def test_unnormalised_input(sre):
    psi = inputs.unnormalised_gaussian_state(9, 3, scale=7.0)
    _check_exact(sre.sre_exact(dev(psi), allow_nullity_error=True), oracle.sre_exact(psi), 9)


# -------------------------------------------------------------- marginal
@pytest.mark.parametrize("N", [1, 2, 5, 10, 13, 14, 16])
def test_marginal_vs_oracle(sre, N):
    psi = inputs.unnormalised_gaussian_state(N, 500 + N)
    p = sre.pauli_x_marginal(dev(psi)).cpu().numpy()
    ref = oracle.x_marginal(psi)
    assert np.max(np.abs(p - ref)) < 1e-12
    assert abs(p.sum() - 1) < 1e-10


def test_marginal_n24_sampled(sre):
    N = 24
    psi = inputs.haar_state(N, 24)
    p = sre.pauli_x_marginal(dev(psi)).cpu().numpy()
    assert abs(p.sum() - 1) < 1e-9
    for x in (0, 1, 12345, (1 << 24) - 1):
        assert abs(p[x] - oracle.x_marginal_one(psi, x)) < 1e-15 + 1e-9 * abs(p[x])


# -------------------------------------------------------------------- MC
@pytest.mark.parametrize("N", [6, 12, 16])
def test_mc_uniform_vs_oracle(sre, N):
    psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 8 * N, 4, 600 + N))
    n_x = 24
    r = sre.sre_mc(dev(psi), sre.SRE_MC_UNIFORM, n_x, 1, seed=11, counter0=3, return_samples=True)
    ref = oracle.mc_uniform(psi, n_x, 11, 3)
    assert np.array_equal(r["xs"].cpu().numpy().astype(np.uint64), ref["xs"])
    assert np.max(np.abs(np.array(r["M"]) - ref["M"])) < TOL_M
    assert np.allclose(r["err_M"], ref["err"], rtol=1e-3, atol=1e-9)


@pytest.mark.parametrize("N,n_x,zpx", [(4, 16, 8), (10, 12, 16), (14, 6, 8), (16, 6, 8)])
def test_mc_marginal_vs_oracle(sre, N, n_x, zpx):
    psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 8 * N, 3, 700 + N))
    r = sre.sre_mc(dev(psi), sre.SRE_MC_MARGINAL, n_x, zpx, seed=21, counter0=0, return_samples=True)
    ref = oracle.mc_marginal(psi, n_x, zpx, 21, 0)
    xs = r["xs"].cpu().numpy().astype(np.uint64)
    zs = r["zs"].cpu().numpy().astype(np.uint64)
    c = r["c"].cpu().numpy()
    assert np.array_equal(xs, ref["xs"])
    assert np.array_equal(zs, ref["zs"])
    assert np.max(np.abs(c - ref["c"])) < TOL_C
    assert np.max(np.abs(np.array(r["M"]) - ref["M"])) < TOL_M
    assert np.max(np.abs(np.array(r["M_rb"]) - ref["M_rb"])) < TOL_M


@pytest.mark.parametrize("N", [12, 16])
def test_mc_marginal_ragged_batches(sre, N):
    """11 families in launches of 4 (4 + 4 + 3): draws, sampled expectations
    and estimates equal the oracle's, as in one launch."""
    psi = oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 8 * N, 3, 720 + N))
    r = sre.sre_mc(dev(psi), sre.SRE_MC_MARGINAL, 11, 8, seed=31, counter0=5, return_samples=True, x_batch=4)
    ref = oracle.mc_marginal(psi, 11, 8, 31, 5)
    assert np.array_equal(r["xs"].cpu().numpy().astype(np.uint64), ref["xs"])
    assert np.array_equal(r["zs"].cpu().numpy().astype(np.uint64), ref["zs"])
    assert np.max(np.abs(r["c"].cpu().numpy() - ref["c"])) < TOL_C
    assert np.max(np.abs(np.array(r["M"]) - ref["M"])) < TOL_M


@pytest.mark.parametrize("N,xb", [(16, 1000), (18, 2999)])
def test_exact_ragged_batches(sre, N, xb):
    """Family batches that do not divide 2^N (a short last launch): the
    per-family sums and their fixed-order totals do not depend on the batch
    size, so M_a and the nullity equal the default plan's exactly."""
    psi = dev(oracle.circuit_state(N, inputs.random_clifford_tdoped_gates(N, 0, 4, 730 + N, n_t=6, first_block=2 * N)))
    # the same tiling in both calls (a process-wide autotuner entry for N
    # would otherwise apply to the call without options only)
    a = sre.sre_exact(psi, radix_log2=13)
    b = sre.sre_exact(psi, radix_log2=13, x_batch=xb)
    assert a["M"] == b["M"] and a["nullity"] == b["nullity"] and a["stab_count"] == b["stab_count"]


def test_mc_is_deterministic_run_to_run(sre):
    N = 17
    psi = dev(inputs.haar_state(N, 3))
    a = sre.sre_mc(psi, sre.SRE_MC_MARGINAL, 40, 32, seed=8, return_samples=True)
    b = sre.sre_mc(psi, sre.SRE_MC_MARGINAL, 40, 32, seed=8, return_samples=True)
    for k in ("xs", "zs", "c"):
        assert torch.equal(a[k], b[k]), k
    assert a["M"] == b["M"] and a["M_rb"] == b["M_rb"]


def test_mc_marginal_stabilizer_exact_zero(sre):
    N = 12
    psi = oracle.circuit_state(N, inputs.random_clifford_gates(N, 96, 41))
    r = sre.sre_mc(dev(psi), sre.SRE_MC_MARGINAL, 32, 16, seed=2, return_samples=True)
    assert np.max(np.abs(r["M"])) < TOL_M and np.max(np.abs(r["M_rb"])) < TOL_M
    assert np.allclose(np.abs(r["c"].cpu().numpy()), 1.0, atol=TOL_C)


def test_mc_n24_full_size_sampled(sre):
    """The headline workload's shape (N=24 Haar, x from p(x), z from the
    family spectrum) on a small x batch: sampled indices against the oracle's
    inverse-CDF draws, sampled c against brute force, M_2 against the Haar
    closed form."""
    N = 24
    psi = inputs.haar_state(N, 24)
    n_x, zpx = 48, 32
    r = sre.sre_mc(dev(psi), sre.SRE_MC_MARGINAL, n_x, zpx, seed=24, return_samples=True)
    xs = r["xs"].cpu().numpy().astype(np.uint64)
    zs = r["zs"].cpu().numpy().astype(np.uint64)
    c = r["c"].cpu().numpy()
    p = oracle.x_marginal(psi)
    p[0] = 0.0                       # families 1.. draw from p(x | x != 0)
    assert xs[0] == 0
    for i in range(1, n_x):
        assert int(xs[i]) == oracle.inverse_cdf(p, oracle.mc_draw(24, 0, i, 0))
    rl = sre.sre_make_plan(N)["range_log2"]
    n_exact = n_total = 0
    for i in (0, 7, 13, 21):
        x = int(xs[i])
        cf = oracle.family_spectrum(psi, x)
        cg = sre.sre_family_spectrum(dev(psi), x).cpu().numpy().astype(np.float64)
        for k in range(zpx):
            u = oracle.mc_draw(24, 0, i, 1 + k)
            zo = oracle.inverse_cdf(cf * cf, u)
            ok, exact = draw_within_bound(int(zs[i, k]), zo, cf * cf, cg * cg, u, rl)
            assert ok, (i, k, int(zs[i, k]), zo)
            n_exact += exact
            n_total += 1
    # Every draw is valid (above). Identity with the FP64 draw is a rate: the
    # FP32 spectrum's running sums differ from the oracle's by ~1e-7 of the
    # total, a few entries of 2^24, so a few percent of draws land 1-7 z
    # later (measured 95-96% identical over 384 draws); 85% of 128 draws is
    # five standard deviations below that.
    assert n_exact >= 0.85 * n_total
    for i, k in ((1, 0), (5, 3), (40, 31)):
        assert abs(c[i, k] - oracle.pauli_expectation(psi, int(xs[i]), int(zs[i, k]))) < TOL_C
    m2_haar = math.log2(2**N + 3) - 2
    assert abs(r["M_rb"][1] - m2_haar) < 4 * r["err_rb"][1] + 1e-4
    assert abs(r["M"][1] - m2_haar) < 5 * r["err_M"][1] + 1e-3


def test_mc_n24_bench_launch_configuration(sre):
    """The benchmark's own configuration: N = 24 Haar (seed 24), 4096 x from
    p(x), 256 z per x, the default plan (128 families per launch, 32 launches
    in the sorted x order). Sampled outputs from the first, a middle and the
    last launch against the oracle: x draws bit-exact, z draws within the
    propagated bound, sampled c against the direct sum; the estimate against
    the Haar closed form."""
    N = 24
    psi = inputs.haar_state(N, 24)
    assert sre.sre_make_plan(N)["x_batch"] == 128
    n_x, zpx = 4096, 256
    r = sre.sre_mc(dev(psi), sre.SRE_MC_MARGINAL, n_x, zpx, seed=24, return_samples=True)
    xs = r["xs"].cpu().numpy().astype(np.uint64)
    zs = r["zs"].cpu().numpy().astype(np.uint64)
    c = r["c"].cpu().numpy()
    p = oracle.x_marginal(psi)
    p[0] = 0.0
    assert xs[0] == 0
    for i in list(range(1, 40)) + list(range(2040, 2060)) + list(range(4070, 4096)):
        assert int(xs[i]) == oracle.inverse_cdf(p, oracle.mc_draw(24, 0, i, 0)), i
    rl = sre.sre_make_plan(N)["range_log2"]
    n_exact = n_total = 0
    for i in (3, 2049, 4095):
        x = int(xs[i])
        cf = oracle.family_spectrum(psi, x)
        cg = sre.sre_family_spectrum(dev(psi), x).cpu().numpy().astype(np.float64)
        for k in range(0, zpx, 8):
            u = oracle.mc_draw(24, 0, i, 1 + k)
            zo = oracle.inverse_cdf(cf * cf, u)
            ok, exact = draw_within_bound(int(zs[i, k]), zo, cf * cf, cg * cg, u, rl)
            assert ok, (i, k, int(zs[i, k]), zo)
            n_exact += exact
            n_total += 1
        for k in (0, 101, 255):
            assert abs(c[i, k] - oracle.pauli_expectation(psi, x, int(zs[i, k]))) < TOL_C
    assert n_exact >= 0.85 * n_total
    m2_haar = math.log2(2**N + 3) - 2
    assert abs(r["M_rb"][1] - m2_haar) < 4 * r["err_rb"][1] + 1e-4


@pytest.mark.parametrize("k_low", [16, 12, 8])
def test_mc_marginal_fine_ranges(sre, k_low):
    """Multi-pass plan (N=16: a 13-bit last pass, z-ranges of 2^10): a Haar
    state on the low k_low qubits with the rest in |0>, so the families' top
    X bit j falls above the last tile (k_low = 16), inside it above the range
    size (12) or below the range size (8) -- the three ways a range maps to
    last-pass outputs. Draws against the oracle's inverse CDF, sampled c
    against brute force."""
    N = 16
    assert sre.sre_make_plan(N)["range_log2"] == 10 and sre.sre_make_plan(N)["pass_bits"][-1] == 13
    psi = np.zeros(1 << N, dtype=np.complex128)
    psi[: 1 << k_low] = inputs.haar_state(k_low, 900 + k_low)
    n_x, zpx = 24, 24
    r = sre.sre_mc(dev(psi), sre.SRE_MC_MARGINAL, n_x, zpx, seed=5, return_samples=True)
    xs = r["xs"].cpu().numpy().astype(np.uint64)
    zs = r["zs"].cpu().numpy().astype(np.uint64)
    c = r["c"].cpu().numpy()
    ref = oracle.mc_marginal(psi, n_x, zpx, 5, 0)
    assert np.array_equal(xs, ref["xs"])
    assert all(int(x) < (1 << k_low) for x in xs)
    ref_zs = ref["zs"].reshape(n_x, zpx)
    n_exact = n_total = 0
    for i in range(n_x):
        x = int(xs[i])
        cf = oracle.family_spectrum(psi, x)
        cg = sre.sre_family_spectrum(dev(psi), x).cpu().numpy().astype(np.float64)
        for k in range(zpx):
            u = oracle.mc_draw(5, 0, i, 1 + k)
            zo = int(ref_zs[i, k])
            assert zo == oracle.inverse_cdf(cf * cf, u)
            ok, exact = draw_within_bound(int(zs[i, k]), zo, cf * cf, cg * cg, u, 10)
            assert ok, (i, k, int(zs[i, k]), zo)
            n_exact += exact
            n_total += 1
            assert abs(c[i, k] - cf[int(zs[i, k])]) < TOL_C
    assert n_exact >= 0.9 * n_total


@pytest.mark.parametrize("radix", [11, 12, 14])
def test_mc_marginal_fold_widths(sre, radix):
    """Last-pass tiles of 2^11, 2^12 and 2^14 points: each draw folds 2, 4
    or 16 blocks of 2^10 outputs through the sampler's bulk-copy ring. Draws
    against the oracle's inverse CDF within the propagated bound, sampled c
    against brute force."""
    N = 16
    plan = sre.sre_make_plan(N, radix_log2=radix)
    assert plan["pass_bits"][-1] == radix and plan["range_log2"] == 10
    psi = inputs.haar_state(N, 950 + radix)
    n_x, zpx = 12, 16
    r = sre.sre_mc(dev(psi), sre.SRE_MC_MARGINAL, n_x, zpx, seed=7, return_samples=True, radix_log2=radix)
    xs = r["xs"].cpu().numpy().astype(np.uint64)
    zs = r["zs"].cpu().numpy().astype(np.uint64).reshape(n_x, zpx)
    c = r["c"].cpu().numpy().reshape(n_x, zpx)
    ref = oracle.mc_marginal(psi, n_x, zpx, 7, 0)
    assert np.array_equal(xs, ref["xs"])
    ref_zs = ref["zs"].reshape(n_x, zpx)
    n_exact = n_total = 0
    for i in range(n_x):
        cf = oracle.family_spectrum(psi, int(xs[i]))
        cg = sre.sre_family_spectrum(dev(psi), int(xs[i]), radix_log2=radix).cpu().numpy().astype(np.float64)
        for k in range(zpx):
            u = oracle.mc_draw(7, 0, i, 1 + k)
            ok, exact = draw_within_bound(int(zs[i, k]), int(ref_zs[i, k]), cf * cf, cg * cg, u, 10)
            assert ok, (i, k, int(zs[i, k]), int(ref_zs[i, k]))
            n_exact += exact
            n_total += 1
            assert abs(c[i, k] - cf[int(zs[i, k])]) < TOL_C
    assert n_exact >= 0.9 * n_total


# ----------------------------------------------------------------- gates
@pytest.mark.parametrize("N,n", [(1, 20), (3, 40), (5, 60), (8, 120), (12, 200), (14, 200), (17, 300)])
def test_gates_vs_oracle(sre, N, n):
    g = np.random.default_rng(N)
    rows = []
    for _ in range(n):
        op = int(g.integers(0, 6)) if N > 1 else int(g.choice([0, 1, 2, 4, 5]))
        q0 = int(g.integers(0, N))
        q1 = int((q0 + 1 + g.integers(0, N - 1)) % N) if op == inputs.GATE_CNOT else 0
        rows.append((op, q0, q1))
    gates = np.array(rows, dtype=np.uint8)
    psi = inputs.haar_state(N, 800 + N)
    want = oracle.apply_gates(psi, gates)
    p = dev(psi)
    sre.apply_clifford_tdoped_circuit(p, gates)
    got = p.cpu().numpy()
    # per amplitude: the 1e-6 target; in l2 norm: the FP32 rounding bound of
    # the gate kernels, 3 u per H or T gate (one add, one multiply and the
    # rounded 1/sqrt2 per output), S and CNOT exact
    d = got - want
    n_ht = int(sum(1 for r in rows if r[0] in (inputs.GATE_H, inputs.GATE_T, inputs.GATE_TDG)))
    assert np.max(np.abs(d)) < 1e-6
    assert np.linalg.norm(d) <= 3 * 2.0**-24 * n_ht * np.linalg.norm(want) + 1e-12


def test_gates_then_exact_matches_oracle_pipeline(sre):
    """The N=10 T-doped workload prepared on the GPU from |0^10>."""
    gates = inputs.workload_n10_states()["tdoped_gates"]
    p = torch.zeros(1 << 10, dtype=torch.complex64, device="cuda")
    p[0] = 1
    sre.apply_clifford_tdoped_circuit(p, gates)
    ref = oracle.sre_exact(oracle.circuit_state(10, gates))
    r = sre.sre_exact(p, allow_nullity_error=True)
    assert np.max(np.abs(np.array(r["M"]) - ref["M"])) < TOL_M
    assert r["nullity"] == ref["nullity"]
