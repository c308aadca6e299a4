"""Seeded synthetic inputs: state vectors and gate lists.

This module is shared by the library's tests, by ``bench.py`` and by the
oracle's tests. It holds none of the method's arithmetic (no Pauli
expectation, no transform, no moment, no sampling of Pauli strings): only
the states and circuits that the method is applied to.

Conventions
-----------
* A state on N qubits is a complex64 vector of length d = 2^N; amplitude
  ``psi[b]`` belongs to the basis state |b>, and qubit j is bit j of b
  (qubit 0 is the least significant bit).
* A gate list is an (n, 3) uint8 array of rows ``(op, q0, q1)``, the same
  packed layout as ``sre_gate`` in ``include/sre.h``. ``q1`` is the CNOT
  target (``q0`` its control) and is 0 for one-qubit gates.

Workloads follow the paper: Haar-random states (main text, "Monte Carlo
sampling with FWHT"), the product magic state |T>^{k} |0>^{N-k} (main text,
"Clifford preconditioning"), and T-doped random Clifford circuits whose
scrambling ratio eta counts Clifford gates per T gate (Eq. eta).
"""
from __future__ import annotations

import numpy as np

# Gate opcodes; they must equal the SRE_GATE_* values in include/sre.h.
GATE_H, GATE_S, GATE_SDG, GATE_CNOT, GATE_T, GATE_TDG = 0, 1, 2, 3, 4, 5
GATE_NAMES = {GATE_H: "H", GATE_S: "S", GATE_SDG: "SDG", GATE_CNOT: "CNOT",
              GATE_T: "T", GATE_TDG: "TDG"}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar_state(N: int, seed: int) -> np.ndarray:
    """Haar-random pure state: i.i.d. complex Gaussian amplitudes, scaled to
    unit norm in float64, then rounded to complex64."""
    g = _rng(seed)
    d = 1 << N
    v = g.standard_normal(d) + 1j * g.standard_normal(d)
    v /= np.sqrt(np.sum(np.abs(v) ** 2))
    return v.astype(np.complex64)


def unnormalised_gaussian_state(N: int, seed: int, scale: float = 3.0) -> np.ndarray:
    """Complex Gaussian amplitudes with no normalisation (norm far from 1),
    for checking that the library normalises the state itself."""
    g = _rng(seed)
    d = 1 << N
    v = scale * (g.standard_normal(d) + 1j * g.standard_normal(d))
    return v.astype(np.complex64)


def basis_state(N: int, b: int = 0) -> np.ndarray:
    v = np.zeros(1 << N, dtype=np.complex64)
    v[b] = 1.0
    return v


def product_state(single_qubit: list) -> np.ndarray:
    """Tensor product of one-qubit states; ``single_qubit[j]`` = (a0, a1) is
    qubit j (bit j of the basis index). Built in complex128, returned as
    complex64."""
    v = np.ones(1, dtype=np.complex128)
    for a0, a1 in single_qubit:           # qubit j becomes the new high bit
        v = np.concatenate([v * a0, v * a1])
    return v.astype(np.complex64)


T_QUBIT = (1 / np.sqrt(2), np.exp(1j * np.pi / 4) / np.sqrt(2))   # |T>
ZERO_QUBIT = (1.0, 0.0)                                            # |0>


def t_product_state(N: int, k: int) -> np.ndarray:
    """|T>^{k} (x) |0>^{N-k}: qubits 0..k-1 carry |T>, the rest |0>."""
    return product_state([T_QUBIT] * k + [ZERO_QUBIT] * (N - k))


def random_product_state(N: int, seed: int) -> np.ndarray:
    """Product of N random one-qubit pure states (uniform on the Bloch sphere)."""
    g = _rng(seed)
    qs = []
    for _ in range(N):
        a = g.standard_normal(2) + 1j * g.standard_normal(2)
        a /= np.linalg.norm(a)
        qs.append((a[0], a[1]))
    return product_state(qs)


def random_clifford_tdoped_gates(N: int, n_clifford: int, eta: int, seed: int,
                                 n_t: int | None = None,
                                 first_block: int = 0) -> np.ndarray:
    """Gate list of a T-doped random Clifford circuit.

    Clifford gates are drawn uniformly from {H_i, S_i, CNOT_ij} (qubits
    uniform; CNOT takes an ordered pair i != j). After every ``eta`` Clifford
    gates one T gate acts on a uniformly random qubit (the scrambling ratio
    of Eq. eta counted in gates). ``first_block`` extra Clifford gates come
    before the first T so the state is already entangled. If ``n_t`` is
    given, the circuit stops after that many T gates (``n_clifford`` is then
    ignored and ``first_block + n_t * eta`` Cliffords are drawn); ``eta <= 0``
    with ``n_t`` is invalid. ``n_t = 0`` gives a pure Clifford circuit of
    ``n_clifford`` gates.
    """
    g = _rng(seed)
    rows = []

    def clifford():
        kind = int(g.integers(0, 3)) if N > 1 else int(g.integers(0, 2))
        if kind == 0:
            rows.append((GATE_H, int(g.integers(0, N)), 0))
        elif kind == 1:
            rows.append((GATE_S, int(g.integers(0, N)), 0))
        else:
            c = int(g.integers(0, N))
            t = int(g.integers(0, N - 1))
            t = t + 1 if t >= c else t
            rows.append((GATE_CNOT, c, t))

    def tgate():
        rows.append((GATE_T, int(g.integers(0, N)), 0))

    for _ in range(first_block):
        clifford()
    if n_t is None:
        for i in range(n_clifford):
            clifford()
            if eta > 0 and (i + 1) % eta == 0:
                tgate()
    else:
        if n_t > 0 and eta <= 0:
            raise ValueError("eta must be positive when n_t > 0")
        if n_t == 0:
            for _ in range(n_clifford):
                clifford()
        for _ in range(n_t):
            for _ in range(eta):
                clifford()
            tgate()
    return np.asarray(rows, dtype=np.uint8).reshape(-1, 3)


def random_clifford_gates(N: int, n_gates: int, seed: int) -> np.ndarray:
    """Uniform random {H, S, CNOT} circuit (no T): a Clifford preconditioner
    or a stabilizer-state preparation from |0^N>."""
    return random_clifford_tdoped_gates(N, n_gates, 0, seed)


# --------------------------------------------- two-qubit gates, brick walls
# A two-qubit gate is a 4x4 complex matrix U[out][in] on an ordered pair of
# qubits (q0, q1); its local basis index is l = bit(q0) + 2 bit(q1), the same
# layout as the matrices apply_two_qubit_gates takes.

def _key(u: np.ndarray) -> tuple:
    """A matrix modulo global phase: divided by the phase of its first entry
    of modulus above 1/4, rounded."""
    f = u.reshape(-1)
    k = int(np.argmax(np.abs(f) > 0.25))
    v = f * (abs(f[k]) / f[k])
    return tuple(np.round(np.concatenate([v.real, v.imag]) * 1e6).astype(np.int64))


_CLIFFORD2 = None


def two_qubit_clifford_table() -> np.ndarray:
    """All 11520 two-qubit Clifford unitaries modulo global phase (complex128,
    (11520, 4, 4)), by breadth-first closure of H and S on either qubit and
    CNOT in both directions."""
    global _CLIFFORD2
    if _CLIFFORD2 is not None:
        return _CLIFFORD2
    h = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    sg = np.diag([1, 1j])
    i2 = np.eye(2)
    cx01 = np.zeros((4, 4)); cx10 = np.zeros((4, 4))
    for l in range(4):
        b0, b1 = l & 1, l >> 1
        cx01[b0 + 2 * (b1 ^ b0), l] = 1      # control q0, target q1
        cx10[(b0 ^ b1) + 2 * b1, l] = 1      # control q1, target q0
    gens = [np.kron(i2, h), np.kron(h, i2), np.kron(i2, sg), np.kron(sg, i2), cx01, cx10]
    seen = {_key(np.eye(4)): np.eye(4, dtype=np.complex128)}
    frontier = [np.eye(4, dtype=np.complex128)]
    while frontier:
        nxt = []
        for u in frontier:
            for g in gens:
                v = g @ u
                k = _key(v)
                if k not in seen:
                    seen[k] = v
                    nxt.append(v)
        frontier = nxt
    _CLIFFORD2 = np.stack(list(seen.values()))
    return _CLIFFORD2


def haar_two_qubit(g: np.random.Generator) -> np.ndarray:
    """Haar-random U(4): QR of a complex Gaussian matrix, R's diagonal phases
    moved into Q."""
    z = (g.standard_normal((4, 4)) + 1j * g.standard_normal((4, 4))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph


def brickwall_circuit(N: int, depth: int, kind: str, seed: int, first_layer: int = 0):
    """Brick-wall circuit of random two-qubit gates on nearest neighbours
    (SM, brick-wall circuits; even and odd layers count separately): layer t
    acts on the pairs (i, i + 1) with i = (t + first_layer) mod 2, i + 2, ...
    kind "clifford": uniform two-qubit Cliffords; "haar": Haar-random U(4).
    Returns (mats complex64 (n, 4, 4), pairs int32 (n, 2))."""
    g = _rng(seed)
    table = two_qubit_clifford_table() if kind == "clifford" else None
    mats, pairs = [], []
    for t in range(depth):
        for i in range((t + first_layer) % 2, N - 1, 2):
            u = table[g.integers(0, len(table))] if table is not None else haar_two_qubit(g)
            mats.append(u)
            pairs.append((i, i + 1))
    if not mats:
        return np.zeros((0, 4, 4), np.complex64), np.zeros((0, 2), np.int32)
    return np.asarray(mats, np.complex64), np.asarray(pairs, np.int32)


def uniform_inputs_u64(n: int, seed: int) -> np.ndarray:
    """Raw 64-bit words for host-side tests of sampling helpers."""
    return _rng(seed).integers(0, 2**63, size=n, dtype=np.int64).astype(np.uint64)


# ---------------------------------------------------------------------------
# Named workloads (the shapes of the paper's experiments)

def workload_n10_states() -> dict:
    """Three N=10 states: (a) Haar, seed 0; (b) T-doped random Clifford
    circuit on |0^10>, 200 Clifford gates with a T after every 10, seed 1
    (as a gate list); (c) |T>^4 (x) |0^6>."""
    return {
        "haar": haar_state(10, 0),
        "tdoped_gates": random_clifford_tdoped_gates(10, 200, 10, 1),
        "t4": t_product_state(10, 4),
    }


def workload_n18_gate_lists() -> list:
    """Twelve N=18 T-doped circuits: eta in {1,4,16} x n_T in {0,8,32,64};
    2N Clifford gates precede the first T; seeds 100+i."""
    out = []
    i = 0
    for eta in (1, 4, 16):
        for n_t in (0, 8, 32, 64):
            gates = random_clifford_tdoped_gates(18, 4 * 18, eta, 100 + i,
                                                 n_t=n_t, first_block=2 * 18)
            out.append({"eta": eta, "n_t": n_t, "seed": 100 + i, "gates": gates})
            i += 1
    return out


def workload_batched_specs(count: int = 4096, seed0: int = 4000,
                           n_min: int = 8, n_max: int = 16) -> list:
    """Uneven batch: N ~ U{n_min..n_max}, eta ~ U{1,2,4,8,32},
    n_T ~ U{1..3N}; state i uses seed seed0+i."""
    out = []
    for i in range(count):
        g = _rng(seed0 + i)
        N = int(g.integers(n_min, n_max + 1))
        eta = int(g.choice([1, 2, 4, 8, 32]))
        n_t = int(g.integers(1, 3 * N + 1))
        out.append({"N": N, "eta": eta, "n_t": n_t, "seed": seed0 + i})
    return out


def batched_gate_list(spec: dict) -> np.ndarray:
    return random_clifford_tdoped_gates(spec["N"], 0, spec["eta"], spec["seed"],
                                        n_t=spec["n_t"], first_block=2 * spec["N"])
