"""FP64 CPU oracle for the FWHT Pauli-spectrum method (test infrastructure).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference leg may import this package. The
library (``paper_2601_00761_gb300``) never imports it, and the two share no
code: the arithmetic lives in ``sre_oracle.c`` (plain C, FP64), compiled
here with gcc into ``liboracle.so`` and called through ctypes.

Each wrapper cites the passage of the paper its C function follows. Parity
pins for every function are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sre_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_c_dp = ctypes.POINTER(ctypes.c_double)
_c_u64p = ctypes.POINTER(ctypes.c_uint64)
_c_fp = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile sre_oracle.c into liboracle.so (gcc, -O2, FP64, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.or_philox4x64_10.argtypes = [_c_u64p, _c_u64p, _c_u64p]
            L.or_u01.argtypes = [ctypes.c_uint64]
            L.or_u01.restype = ctypes.c_double
            L.or_mc_uniform_draw.argtypes = [ctypes.c_uint64] * 4
            L.or_mc_uniform_draw.restype = ctypes.c_double
            L.or_norm2.argtypes = [_c_fp, ctypes.c_int]
            L.or_norm2.restype = ctypes.c_double
            L.or_pauli_expectation.argtypes = [_c_fp, ctypes.c_int, ctypes.c_uint64,
                                               ctypes.c_uint64, _c_dp]
            L.or_pauli_expectation.restype = ctypes.c_double
            L.or_fwht_real.argtypes = [_c_dp, ctypes.c_int]
            L.or_family_spectrum.argtypes = [_c_fp, ctypes.c_int, ctypes.c_uint64,
                                             ctypes.c_double, _c_dp, _c_dp, ctypes.c_void_p]
            L.or_family_spectrum.restype = ctypes.c_int
            L.or_sre_exact.argtypes = [_c_fp, ctypes.c_int, ctypes.c_double, _c_dp, _c_dp,
                                       ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_int), _c_dp]
            L.or_sre_exact.restype = ctypes.c_int
            L.or_sre_bruteforce.argtypes = [_c_fp, ctypes.c_int, ctypes.c_double, _c_dp, _c_dp,
                                            ctypes.POINTER(ctypes.c_longlong)]
            L.or_sre_bruteforce.restype = ctypes.c_int
            L.or_x_marginal_direct.argtypes = [_c_fp, ctypes.c_int, _c_dp]
            L.or_x_marginal_one.argtypes = [_c_fp, ctypes.c_int, ctypes.c_uint64]
            L.or_x_marginal_one.restype = ctypes.c_double
            L.or_x_marginal_wht.argtypes = [_c_fp, ctypes.c_int, _c_dp]
            L.or_x_marginal_wht.restype = ctypes.c_int
            L.or_inverse_cdf.argtypes = [_c_dp, ctypes.c_uint64, ctypes.c_double]
            L.or_inverse_cdf.restype = ctypes.c_uint64
            L.or_mc_uniform.argtypes = [_c_fp, ctypes.c_int, ctypes.c_longlong, ctypes.c_uint64,
                                        ctypes.c_uint64, _c_dp, _c_dp, _c_u64p]
            L.or_mc_uniform.restype = ctypes.c_int
            L.or_mc_marginal.argtypes = [_c_fp, ctypes.c_int, ctypes.c_longlong, ctypes.c_int,
                                         ctypes.c_uint64, ctypes.c_uint64, _c_dp, _c_dp, _c_dp,
                                         _c_dp, _c_u64p, _c_u64p, _c_dp]
            L.or_mc_marginal.restype = ctypes.c_int
            L.or_apply_gates.argtypes = [_c_dp, ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong]
            L.or_apply_gates.restype = ctypes.c_int
            L.or_set_mutation.argtypes = [ctypes.c_int]
            L.or_exact_families.argtypes = [_c_fp, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                            ctypes.c_uint64, _c_dp, ctypes.c_void_p]
            L.or_exact_finalize.argtypes = [_c_dp, ctypes.c_void_p, ctypes.c_int, _c_dp, _c_dp,
                                            ctypes.c_void_p, ctypes.c_void_p]
            L.or_exact_finalize.restype = None
            L.or_fluctuation_ratio.argtypes = [_c_fp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
            L.or_apply_two_qubit.argtypes = [_c_dp, ctypes.c_int, _c_dp, ctypes.c_void_p, ctypes.c_longlong]
            L.or_apply_two_qubit.restype = ctypes.c_int
            L.or_sre_mixed.argtypes = [_c_fp, ctypes.c_int, ctypes.c_int, _c_dp, _c_dp,
                                       ctypes.POINTER(ctypes.c_double)]
            L.or_sre_mixed.restype = ctypes.c_int
            L.or_sre_mixed_bruteforce.argtypes = [_c_fp, ctypes.c_int, ctypes.c_int, _c_dp, _c_dp,
                                                  ctypes.POINTER(ctypes.c_double)]
            L.or_sre_mixed_bruteforce.restype = None
            L.or_fluctuation_ratio.restype = ctypes.c_int
            L.or_clifford_conjugate.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_uint64,
                                                ctypes.c_uint64, _c_u64p, _c_u64p, ctypes.POINTER(ctypes.c_int)]
            L.or_clifford_conjugate.restype = ctypes.c_int
            _lib = L
    return _lib


def _psi(psi) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(psi, dtype=np.complex64))
    return a


def _fp(a: np.ndarray):
    return a.ctypes.data_as(_c_fp)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_c_dp)


def _nq(psi: np.ndarray) -> int:
    N = int(psi.size).bit_length() - 1
    if psi.size != (1 << N):
        raise ValueError("state length must be a power of two")
    return N


def set_mutation(m: int) -> None:
    """Plant mistake ``m`` in the oracle (0 = none); used only by tests that
    show each pin catches a plausible mistake."""
    lib().or_set_mutation(int(m))


def philox4x64_10(ctr, key) -> np.ndarray:
    """Philox4x64-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(c.ctypes.data_as(_c_u64p), k.ctypes.data_as(_c_u64p),
                           out.ctypes.data_as(_c_u64p))
    return out


def u01(w: int) -> float:
    return lib().or_u01(int(w))


def mc_draw(seed: int, ctr0: int, i: int, lane: int) -> float:
    """Uniform of the sre_mc streams: lane 0 is the x draw of family i,
    lane 1+k its k-th z draw."""
    return lib().or_mc_uniform_draw(int(seed), int(ctr0), int(i), int(lane))


def norm2(psi) -> float:
    a = _psi(psi)
    return lib().or_norm2(_fp(a), _nq(a))


def pauli_expectation(psi, x: int, z: int, return_imag: bool = False):
    """c_{x,z} by the direct O(d) sum of Eq. Pxz-corr."""
    a = _psi(psi)
    im = ctypes.c_double(0.0)
    re = lib().or_pauli_expectation(_fp(a), _nq(a), int(x), int(z), ctypes.byref(im))
    return (re, im.value) if return_imag else re


def all_expectations_bruteforce(psi) -> np.ndarray:
    """c[x, z] for all 4^N strings by brute force (O(8^N); N <= 8)."""
    a = _psi(psi)
    N = _nq(a)
    d = 1 << N
    out = np.empty((d, d))
    for x in range(d):
        for z in range(d):
            out[x, z] = pauli_expectation(a, x, z)
    return out


def family_spectrum(psi, x: int, return_imag: bool = False):
    """c_{x,z} for all z by one FWHT of f_x (Algorithm 1, loop body)."""
    a = _psi(psi)
    N = _nq(a)
    s = 1.0 / norm2(a)
    c = np.empty(1 << N)
    im = ctypes.c_double(0.0)
    rc = lib().or_family_spectrum(_fp(a), N, int(x), s, _dp(c), ctypes.byref(im), None)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return (c, im.value) if return_imag else c


def fwht_real(v) -> np.ndarray:
    a = np.array(v, dtype=np.float64, copy=True)
    n = int(a.size).bit_length() - 1
    lib().or_fwht_real(_dp(a), n)
    return a


def sre_exact(psi, eps: float = 1e-6, per_family: bool = False) -> dict:
    """Algorithm 1: M_1, M_2, M_3 and the nullity from all 4^N correlators."""
    a = _psi(psi)
    N = _nq(a)
    M = np.zeros(3)
    S = np.zeros(3)
    cnt = ctypes.c_longlong(0)
    nul = ctypes.c_int(0)
    fam = np.zeros((1 << N, 4)) if per_family else None
    rc = lib().or_sre_exact(_fp(a), N, eps, _dp(M), _dp(S), ctypes.byref(cnt),
                            ctypes.byref(nul), _dp(fam) if fam is not None else None)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    out = {"M": M, "S": S, "stab_count": cnt.value, "nullity": nul.value}
    if fam is not None:
        out["family"] = fam
    return out


def exact_families(psi, x0: int, x1: int, eps: float = 1e-6):
    """Algorithm 1's loop body for x0 <= x < x1: per-family sums
    [sum c^2, sum c^4, sum c^6, sum c^2 log2 c^2] (shape (x1-x0, 4)) and counts
    of | |c| - 1 | < eps. Families are independent; exact_finalize sums them."""
    a = _psi(psi)
    N = _nq(a)
    fam = np.zeros((x1 - x0, 4))
    cnt = np.zeros(x1 - x0, dtype=np.int64)
    rc = lib().or_exact_families(_fp(a), N, eps, x0, x1, _dp(fam),
                                 cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    if rc != 0:
        raise ValueError("or_exact_families failed")
    return fam, cnt


def exact_finalize(fam, cnt, N: int) -> dict:
    """M_1..M_3, S, stabilizer count and nullity from all d families' sums (x order)."""
    fam = np.ascontiguousarray(fam, dtype=np.float64)
    cnt = np.ascontiguousarray(cnt, dtype=np.int64)
    assert fam.shape == (1 << N, 4) and cnt.shape == (1 << N,)
    M = np.zeros(3)
    S = np.zeros(3)
    sc = ctypes.c_longlong(0)
    nul = ctypes.c_int(0)
    lib().or_exact_finalize(_dp(fam), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), N, _dp(M), _dp(S),
                            ctypes.byref(sc), ctypes.byref(nul))
    return {"M": M, "S": S, "stab_count": sc.value, "nullity": nul.value}


def apply_two_qubit(psi, mats, pairs) -> np.ndarray:
    """The state after the two-qubit gates (mats (n, 4, 4) U[out][in], local
    index bit(q0) + 2 bit(q1); pairs (n, 2) = (q0, q1)), in complex128."""
    v = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128)).copy()
    N = int(round(math.log2(v.size)))
    m = np.ascontiguousarray(np.asarray(mats, dtype=np.complex128).reshape(-1, 4, 4))
    mm = np.ascontiguousarray(np.stack([m.real, m.imag], axis=-1).reshape(-1))
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    rc = lib().or_apply_two_qubit(v.ctypes.data_as(_c_dp), N, mm.ctypes.data_as(_c_dp),
                                  pr.ctypes.data_as(ctypes.c_void_p), pr.shape[0])
    if rc != 0:
        raise ValueError("bad qubit pair")
    return v


def sre_mixed(psi, NA: int, route: str = "partial") -> dict:
    """SRE of the reduced state on the first NA qubits (SM, mixed states):
    {"W": sums over P_A of c^2, c^4, c^6, c^2 log2 c^2, "S2": S_2(rho_A),
    "M": [M_1 (NaN unless rho_A is pure), M_2, M_3]}. route "partial": the
    SM's partial sums + one NA-bit transform per x_A; "bruteforce": every
    P in P_A by its direct correlator."""
    a = _psi(psi)
    N = _nq(a)
    if not 1 <= NA <= N:
        raise ValueError("NA outside 1..N")
    W, M = np.zeros(4), np.zeros(3)
    S2 = ctypes.c_double(0.0)
    if route == "partial":
        if lib().or_sre_mixed(_fp(a), N, NA, _dp(W), _dp(M), ctypes.byref(S2)) != 0:
            raise MemoryError("oracle allocation failed")
    else:
        lib().or_sre_mixed_bruteforce(_fp(a), N, NA, _dp(W), _dp(M), ctypes.byref(S2))
    return {"W": W, "S2": S2.value, "M": M}


def fluctuation_ratio(psi) -> float:
    """r_2 = Std_{x != 0}(m_{2;x}) / E_x[m_{2;x}] over all X-masks (SM,
    Clifford preconditioning), m_{2;x} from the family's FP64 spectrum."""
    a = _psi(psi)
    r = ctypes.c_double(0.0)
    if lib().or_fluctuation_ratio(_fp(a), _nq(a), ctypes.byref(r)) != 0:
        raise MemoryError("oracle allocation failed")
    return r.value


def sre_bruteforce(psi, eps: float = 1e-6) -> dict:
    a = _psi(psi)
    N = _nq(a)
    M = np.zeros(3)
    S = np.zeros(3)
    cnt = ctypes.c_longlong(0)
    lib().or_sre_bruteforce(_fp(a), N, eps, _dp(M), _dp(S), ctypes.byref(cnt))
    return {"M": M, "S": S, "stab_count": cnt.value}


def x_marginal(psi, route: str = "wht") -> np.ndarray:
    a = _psi(psi)
    N = _nq(a)
    p = np.zeros(1 << N)
    if route == "direct":
        lib().or_x_marginal_direct(_fp(a), N, _dp(p))
    else:
        lib().or_x_marginal_wht(_fp(a), N, _dp(p))
    return p


def x_marginal_one(psi, x: int) -> float:
    """p(x) for one x by the direct O(d) sum (Parseval on f_x)."""
    a = _psi(psi)
    return lib().or_x_marginal_one(_fp(a), _nq(a), int(x))


def inverse_cdf(w, u: float) -> int:
    a = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    return int(lib().or_inverse_cdf(_dp(a), a.size, float(u)))


def mc_uniform(psi, n_x: int, seed: int, ctr0: int = 0) -> dict:
    a = _psi(psi)
    N = _nq(a)
    M = np.zeros(3)
    err = np.zeros(3)
    xs = np.zeros(n_x, dtype=np.uint64)
    rc = lib().or_mc_uniform(_fp(a), N, n_x, seed, ctr0, _dp(M), _dp(err),
                             xs.ctypes.data_as(_c_u64p))
    if rc != 0:
        raise ValueError("or_mc_uniform failed")
    return {"M": M, "err": err, "xs": xs}


def mc_marginal(psi, n_x: int, z_per_x: int, seed: int, ctr0: int = 0) -> dict:
    a = _psi(psi)
    N = _nq(a)
    M, err, Mrb, errb = (np.zeros(3) for _ in range(4))
    xs = np.zeros(n_x, dtype=np.uint64)
    zs = np.zeros(n_x * z_per_x, dtype=np.uint64)
    cs = np.zeros(n_x * z_per_x)
    rc = lib().or_mc_marginal(_fp(a), N, n_x, z_per_x, seed, ctr0, _dp(M), _dp(err),
                              _dp(Mrb), _dp(errb), xs.ctypes.data_as(_c_u64p),
                              zs.ctypes.data_as(_c_u64p), _dp(cs))
    if rc != 0:
        raise ValueError("or_mc_marginal failed")
    return {"M": M, "err": err, "M_rb": Mrb, "err_rb": errb, "xs": xs,
            "zs": zs.reshape(n_x, z_per_x), "c": cs.reshape(n_x, z_per_x)}


def apply_gates(psi, gates, N: int | None = None) -> np.ndarray:
    """Apply a gate list (rows op, q0, q1) in FP64; returns complex128."""
    a = np.array(psi, dtype=np.complex128, copy=True)
    N = _nq(a) if N is None else N
    g = np.ascontiguousarray(np.asarray(gates, dtype=np.uint8).reshape(-1, 3))
    rc = lib().or_apply_gates(a.view(np.float64).ctypes.data_as(_c_dp), N,
                              g.ctypes.data, g.shape[0])
    if rc != 0:
        raise ValueError("bad gate row")
    return a


def clifford_conjugate(N: int, gates, x: int, z: int):
    """(x', z', sign) with C^dag P_{x,z} C = sign * P_{x',z'} for the Clifford
    gate list C (applied in list order); raises on a T gate."""
    g = np.ascontiguousarray(np.asarray(gates, dtype=np.uint8).reshape(-1, 3))
    xo = ctypes.c_uint64(0)
    zo = ctypes.c_uint64(0)
    sg = ctypes.c_int(0)
    rc = lib().or_clifford_conjugate(N, g.ctypes.data, g.shape[0], int(x), int(z), ctypes.byref(xo),
                                     ctypes.byref(zo), ctypes.byref(sg))
    if rc != 0:
        raise ValueError("not a Clifford gate list")
    return xo.value, zo.value, sg.value


def circuit_state(N: int, gates) -> np.ndarray:
    """|0^N> after the gate list, in FP64, rounded to complex64 (the input
    both sides receive when a test starts from a circuit)."""
    psi = np.zeros(1 << N, dtype=np.complex128)
    psi[0] = 1.0
    return apply_gates(psi, gates, N).astype(np.complex64)
