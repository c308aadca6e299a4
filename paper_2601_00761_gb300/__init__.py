"""GB300 (sm_103a) library for the FWHT Pauli-spectrum method of Xiao & Ryu,
"Exponentially Accelerated Sampling of Pauli Strings for Nonstabilizerness"
(arXiv 2601.00761).

This module is a thin ctypes binding over the C ABI declared in
``include/sre.h`` (``libsre.so``, built by ``paper_2601_00761_gb300.build``).
It only marshals arguments: every step of the computation runs in the
library's CUDA kernels. Tensors are PyTorch tensors on the current CUDA
device; work is issued on PyTorch's current stream. If ``libsre.so`` is
missing the import of any entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["sre_version", "sre_last_error", "sre_default_opts", "sre_make_plan", "sre_workspace_bytes",
           "sre_release_workspace", "sre_norm2", "sre_exact", "sre_exact_batched", "sre_mc",
           "pauli_x_marginal", "stabilizer_nullity", "apply_clifford_tdoped_circuit",
           "sre_family_spectrum", "sre_family_spectrum_f64", "sre_philox_blocks", "sre_kernel_launches", "sre_device_allocations", "sre_tc_gemm_selftest",
           "sre_selftest_bounded_wait", "sre_selftest_queue_wait",
           "sre_profile_passes", "sre_pass_timing", "sre_exact_noalloc", "sre_autotune", "sre_autotune_clear", "SreError",
           "SRE_FP32_SIMT", "SRE_BF16X2_TC", "SRE_BF16X3_TC", "SRE_MC_UNIFORM", "SRE_MC_MARGINAL",
           "lib_path", "load"]

_PKG = os.path.dirname(os.path.abspath(__file__))
# SRE_LIBRARY selects another build of the same library (e.g. a tuning variant)
_LIB_PATH = os.environ.get("SRE_LIBRARY") or os.path.join(_PKG, "libsre.so")

SRE_OK, SRE_EINVAL, SRE_ENOMEM, SRE_ECUDA, SRE_EZERO, SRE_ENULLITY, SRE_ETIMEOUT, SRE_ENOTSUP = range(8)
STATUS_NAMES = {0: "SRE_OK", 1: "SRE_EINVAL", 2: "SRE_ENOMEM", 3: "SRE_ECUDA", 4: "SRE_EZERO",
                5: "SRE_ENULLITY", 6: "SRE_ETIMEOUT", 7: "SRE_ENOTSUP"}
SRE_FP32_SIMT, SRE_BF16X2_TC, SRE_BF16X3_TC = 0, 1, 2
SRE_MC_UNIFORM, SRE_MC_MARGINAL = 0, 1


class SreError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("eps_null", ctypes.c_double), ("radix_log2", ctypes.c_int),
                ("tile_log2", ctypes.c_int), ("x_batch", ctypes.c_int), ("batch_queue", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("M", ctypes.c_double * 3), ("S", ctypes.c_double * 3), ("err_M", ctypes.c_double * 3),
                ("M_rb", ctypes.c_double * 3), ("err_rb", ctypes.c_double * 3), ("parseval", ctypes.c_double),
                ("stab_count", ctypes.c_longlong), ("nullity", ctypes.c_int), ("n_passes", ctypes.c_int),
                ("n_flagged", ctypes.c_longlong), ("n_families", ctypes.c_longlong),
                ("n_samples", ctypes.c_longlong), ("n_boundary", ctypes.c_longlong), ("r2", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {"M": list(self.M), "S": list(self.S), "err_M": list(self.err_M), "M_rb": list(self.M_rb),
                "err_rb": list(self.err_rb), "parseval": self.parseval, "stab_count": self.stab_count,
                "nullity": self.nullity, "n_passes": self.n_passes, "n_flagged": self.n_flagged,
                "n_families": self.n_families, "n_samples": self.n_samples, "r2": self.r2}


class MixedResult(ctypes.Structure):
    _fields_ = [("M", ctypes.c_double * 3), ("S2", ctypes.c_double), ("W", ctypes.c_double * 4),
                ("err_M", ctypes.c_double * 3), ("N_A", ctypes.c_int)]


class Plan(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("n_bits", ctypes.c_int), ("n_passes", ctypes.c_int),
                ("pass_lo", ctypes.c_int * 4), ("pass_bits", ctypes.c_int * 4), ("x_batch", ctypes.c_int),
                ("range_log2", ctypes.c_int), ("workspace_exact", ctypes.c_size_t)]


class Gate(ctypes.Structure):
    _pack_ = 1
    _fields_ = [("op", ctypes.c_ubyte), ("q0", ctypes.c_ubyte), ("q1", ctypes.c_ubyte)]


_lib = None
_vp = ctypes.c_void_p


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libsre.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with `python -m paper_2601_00761_gb300.build`")
    L = ctypes.CDLL(_LIB_PATH)
    st = ctypes.c_int
    sig = {
        "sre_version": ([], ctypes.c_char_p),
        "sre_last_error": ([], ctypes.c_char_p),
        "sre_default_opts": ([ctypes.POINTER(Opts)], None),
        "sre_make_plan": ([ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(Plan)], st),
        "sre_workspace_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_int,
                                 ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_size_t)], st),
        "sre_release_workspace": ([], st),
        "sre_norm2": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp], st),
        "sre_exact": ([_vp, ctypes.c_int, ctypes.POINTER(Opts), _vp, ctypes.c_size_t, _vp,
                       ctypes.POINTER(Result)], st),
        "sre_exact_batched": ([ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                               ctypes.POINTER(Opts), _vp, ctypes.c_size_t, _vp, ctypes.POINTER(Result)], st),
        "sre_mc": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_ulonglong,
                    ctypes.c_ulonglong, ctypes.POINTER(Opts), _vp, ctypes.c_size_t, _vp,
                    ctypes.POINTER(Result), _vp, _vp, _vp], st),
        "pauli_x_marginal": ([_vp, ctypes.c_int, _vp, _vp, ctypes.c_size_t, _vp], st),
        "stabilizer_nullity": ([_vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_longlong), _vp], st),
        "apply_clifford_tdoped_circuit": ([_vp, ctypes.c_int, _vp, ctypes.c_longlong, _vp], st),
        "apply_two_qubit_gates": ([_vp, ctypes.c_int, _vp, _vp, ctypes.c_longlong, _vp], st),
        "sre_mixed_workspace_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)], st),
        "sre_mixed": ([_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(MixedResult)], st),
        "sre_family_spectrum": ([_vp, ctypes.c_int, ctypes.c_ulonglong, ctypes.POINTER(Opts), _vp, _vp], st),
        "sre_family_spectrum_f64": ([_vp, ctypes.c_int, ctypes.c_ulonglong, _vp, _vp], st),
        "sre_philox_blocks": ([_vp, _vp, ctypes.c_int, _vp], st),
        "sre_kernel_launches": ([], ctypes.c_ulonglong),
        "sre_device_allocations": ([], ctypes.c_ulonglong),
        "sre_tc_gemm_selftest": ([_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp],
                                 st),
        "sre_selftest_bounded_wait": ([_vp], st),
        "sre_selftest_queue_wait": ([_vp], st),
        "sre_autotune": ([_vp, ctypes.c_int, _vp, ctypes.POINTER(Opts)], st),
        "sre_autotune_clear": ([ctypes.c_int], st),
        "sre_exact_noalloc": ([_vp, ctypes.c_int, ctypes.POINTER(Opts), _vp, ctypes.POINTER(Result)], st),
        "sre_pass_timing": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_double)], st),
        "sre_profile_passes": ([_vp, ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(Opts), _vp,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(status: int, allow=()):
    if status != SRE_OK and status not in allow:
        raise SreError(status, load().sre_last_error().decode())
    return status


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _psi_ptr(psi, N=None):
    torch = _torch()
    if not isinstance(psi, torch.Tensor) or not psi.is_cuda:
        raise TypeError("psi must be a CUDA tensor")
    if psi.dtype != torch.complex64 or not psi.is_contiguous():
        raise TypeError("psi must be a contiguous complex64 tensor")
    n = psi.numel()
    Nq = n.bit_length() - 1
    if n != 1 << Nq:
        raise ValueError("psi length must be a power of two")
    if N is not None and N != Nq:
        raise ValueError("N does not match psi")
    return ctypes.c_void_p(psi.data_ptr()), Nq


def _opts(precision=SRE_FP32_SIMT, eps_null=1e-6, radix_log2=0, tile_log2=0, x_batch=0, batch_queue=0, opts=None):
    if opts is not None:
        return opts
    o = Opts()
    load().sre_default_opts(ctypes.byref(o))
    o.precision, o.eps_null, o.radix_log2, o.tile_log2, o.x_batch = precision, eps_null, radix_log2, tile_log2, x_batch
    o.batch_queue = batch_queue
    return o


def sre_version() -> str:
    return load().sre_version().decode()


def sre_last_error() -> str:
    return load().sre_last_error().decode()


def sre_default_opts() -> Opts:
    o = Opts()
    load().sre_default_opts(ctypes.byref(o))
    return o


def sre_make_plan(N: int, **kw) -> dict:
    p = Plan()
    _check(load().sre_make_plan(N, ctypes.byref(_opts(**kw)), ctypes.byref(p)))
    return {"N": p.N, "n_bits": p.n_bits, "n_passes": p.n_passes, "pass_lo": list(p.pass_lo)[:p.n_passes],
            "pass_bits": list(p.pass_bits)[:p.n_passes], "x_batch": p.x_batch, "range_log2": p.range_log2,
            "workspace_exact": p.workspace_exact}


def sre_workspace_bytes(N: int, mode: int = -1, n_x: int = 0, z_per_x: int = 0, **kw) -> int:
    b = ctypes.c_size_t(0)
    _check(load().sre_workspace_bytes(N, mode, n_x, z_per_x, ctypes.byref(_opts(**kw)), ctypes.byref(b)))
    return b.value


def sre_release_workspace() -> None:
    _check(load().sre_release_workspace())


def _workspace(workspace):
    if workspace is None:
        return None, 0
    return ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()


def sre_norm2(psi) -> float:
    p, N = _psi_ptr(psi)
    out = ctypes.c_double(0)
    _check(load().sre_norm2(p, N, ctypes.byref(out), _stream()))
    return out.value


def sre_exact(psi, workspace=None, allow_nullity_error=False, **kw) -> dict:
    """Algorithm 1 over all 4^N strings: M_1, M_2, M_3 and the nullity."""
    p, N = _psi_ptr(psi)
    r = Result()
    ws, wb = _workspace(workspace)
    st = load().sre_exact(p, N, ctypes.byref(_opts(**kw)), ws, wb, _stream(), ctypes.byref(r))
    _check(st, allow=(SRE_ENULLITY,) if allow_nullity_error else ())
    d = r.as_dict()
    d["status"] = st
    return d


def sre_autotune(psi) -> dict:
    """Pick the fastest tiling for psi's N (kept for later calls)."""
    p, N = _psi_ptr(psi)
    o = Opts()
    _check(load().sre_autotune(p, N, _stream(), ctypes.byref(o)))
    return {"radix_log2": o.radix_log2, "tile_log2": o.tile_log2, "x_batch": o.x_batch}


def sre_autotune_clear(N: int = 0) -> None:
    """Drop the autotuner's choice for N (0: every N); plans return to the defaults."""
    _check(load().sre_autotune_clear(N))


def sre_exact_batched(psis, **kw) -> list:
    ptrs, Ns = [], []
    for psi in psis:
        p, N = _psi_ptr(psi)
        ptrs.append(p.value)
        Ns.append(N)
    cnt = len(ptrs)
    P = (_vp * cnt)(*ptrs)
    Nn = (ctypes.c_int * cnt)(*Ns)
    R = (Result * cnt)()
    _check(load().sre_exact_batched(P, Nn, cnt, ctypes.byref(_opts(**kw)), None, 0, _stream(), R))
    return [R[i].as_dict() for i in range(cnt)]


def sre_mc(psi, mode: int = SRE_MC_MARGINAL, n_x: int = 4096, z_per_x: int = 256, seed: int = 0,
           counter0: int = 0, workspace=None, return_samples: bool = False, outputs=None, **kw) -> dict:
    """Monte Carlo over X-mask families (SM Sec. I estimator, or x from the
    exact marginal with z from the family spectrum)."""
    torch = _torch()
    p, N = _psi_ptr(psi)
    r = Result()
    ws, wb = _workspace(workspace)
    xs = zs = cs = None
    if outputs is not None:
        xs, zs, cs = outputs
    elif return_samples:
        dev = psi.device
        xs = torch.empty(n_x, dtype=torch.int64, device=dev)
        if mode == SRE_MC_MARGINAL:
            zs = torch.empty(n_x * z_per_x, dtype=torch.int64, device=dev)
            cs = torch.empty(n_x * z_per_x, dtype=torch.float32, device=dev)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    _check(load().sre_mc(p, N, mode, n_x, z_per_x, seed, counter0, ctypes.byref(_opts(**kw)), ws, wb, _stream(),
                         ctypes.byref(r), ptr(xs), ptr(zs), ptr(cs)))
    d = r.as_dict()
    if return_samples or outputs is not None:
        d["xs"] = xs
        d["zs"] = zs.view(n_x, z_per_x) if zs is not None else None
        d["c"] = cs.view(n_x, z_per_x) if cs is not None else None
    return d


def pauli_x_marginal(psi, out=None, workspace=None):
    """p(x) = sum_z c_{x,z}^2 / d for every x (float64 tensor of length d)."""
    torch = _torch()
    p, N = _psi_ptr(psi)
    if out is None:
        out = torch.empty(1 << N, dtype=torch.float64, device=psi.device)
    ws, wb = _workspace(workspace)
    _check(load().pauli_x_marginal(p, N, ctypes.c_void_p(out.data_ptr()), ws, wb, _stream()))
    return out


def stabilizer_nullity(psi, eps: float = 1e-6, allow_nullity_error=False):
    p, N = _psi_ptr(psi)
    nu = ctypes.c_int(-1)
    cnt = ctypes.c_longlong(-1)
    _check(load().stabilizer_nullity(p, N, eps, ctypes.byref(nu), ctypes.byref(cnt), _stream()),
           allow=(SRE_ENULLITY,) if allow_nullity_error else ())
    return nu.value, cnt.value


def apply_clifford_tdoped_circuit(psi, gates) -> None:
    """Apply gate rows (op, q0, q1) in order, in place."""
    p, N = _psi_ptr(psi)
    g = np.ascontiguousarray(np.asarray(gates, dtype=np.uint8).reshape(-1, 3))
    _check(load().apply_clifford_tdoped_circuit(p, N, g.ctypes.data_as(ctypes.c_void_p), g.shape[0], _stream()))


def sre_mixed_workspace_bytes(N: int, N_A: int) -> int:
    b = ctypes.c_size_t(0)
    _check(load().sre_mixed_workspace_bytes(N, N_A, ctypes.byref(b)))
    return b.value


def sre_mixed(psi, N_A: int, workspace=None) -> dict:
    """SRE of the reduced state on the first N_A qubits (SM, mixed states):
    {"M": [M_1 (NaN unless rho_A is pure), M_2, M_3], "S2", "W", "err_M"}."""
    p, N = _psi_ptr(psi)
    r = MixedResult()
    ws, wb = _workspace(workspace)
    _check(load().sre_mixed(p, N, N_A, ws, wb, _stream(), ctypes.byref(r)))
    return {"M": list(r.M), "S2": r.S2, "W": list(r.W), "err_M": list(r.err_M), "N_A": r.N_A}


def apply_two_qubit_gates(psi, mats, pairs) -> None:
    """Apply 4x4 gates in order, in place: mats (n, 4, 4) complex U[out][in]
    with local index bit(q0) + 2 bit(q1), pairs (n, 2) = (q0, q1)."""
    p, N = _psi_ptr(psi)
    m = np.asarray(mats, dtype=np.complex64).reshape(-1, 4, 4)
    mm = np.ascontiguousarray(np.stack([m.real, m.imag], axis=-1).astype(np.float32).reshape(-1))
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    if pr.shape[0] != m.shape[0]:
        raise ValueError("one qubit pair per matrix")
    _check(load().apply_two_qubit_gates(p, N, mm.ctypes.data_as(ctypes.c_void_p), pr.ctypes.data_as(ctypes.c_void_p),
                                        pr.shape[0], _stream()))


def sre_family_spectrum(psi, x: int, out=None, **kw):
    """c_{x,z} for all z (float32)."""
    torch = _torch()
    p, N = _psi_ptr(psi)
    if out is None:
        out = torch.empty(1 << N, dtype=torch.float32, device=psi.device)
    _check(load().sre_family_spectrum(p, N, x, ctypes.byref(_opts(**kw)), ctypes.c_void_p(out.data_ptr()),
                                      _stream()))
    return out


def sre_family_spectrum_f64(psi, x: int, out=None):
    torch = _torch()
    p, N = _psi_ptr(psi)
    if out is None:
        out = torch.empty(1 << N, dtype=torch.float64, device=psi.device)
    _check(load().sre_family_spectrum_f64(p, N, x, ctypes.c_void_p(out.data_ptr()), _stream()))
    return out


def sre_philox_blocks(ctr_key):
    """Philox4x64-10 blocks of the device generator: ctr_key (n, 6) int64
    CUDA tensor of (c0, c1, c2, c3, k0, k1) rows -> (n, 4) words."""
    torch = _torch()
    n = ctr_key.shape[0]
    out = torch.empty((n, 4), dtype=torch.int64, device=ctr_key.device)
    _check(load().sre_philox_blocks(ctypes.c_void_p(ctr_key.data_ptr()), ctypes.c_void_p(out.data_ptr()), n,
                                    _stream()))
    return out


def sre_selftest_queue_wait() -> int:
    """Run the persistent-queue wait self-test on the current stream; returns
    the status (SRE_ETIMEOUT when the bound works)."""
    return int(load().sre_selftest_queue_wait(_stream()))


def sre_selftest_bounded_wait() -> int:
    """Run the bounded-wait self-test on the current stream; returns the
    status (SRE_ETIMEOUT when the bound works)."""
    return int(load().sre_selftest_bounded_wait(_stream()))


def sre_kernel_launches() -> int:
    """Kernels the library has launched since it was loaded."""
    return int(load().sre_kernel_launches())


def sre_tc_gemm_selftest(A, B, swizzle: int = 128):
    """D = A B^T (FP32) from BF16 device matrices A (M x K) and B (N x K)
    through the library's tcgen05 self-test kernel."""
    import torch
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and A.is_contiguous() and B.is_contiguous()
    M, K = A.shape
    N = B.shape[0]
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(load().sre_tc_gemm_selftest(_vp(A.data_ptr()), _vp(B.data_ptr()), _vp(D.data_ptr()), M, N, K, swizzle,
                                       _vp(err.data_ptr()), _stream()))
    return D


def sre_device_allocations() -> int:
    """Device allocations (cudaMalloc) the library has made since it was loaded."""
    return int(load().sre_device_allocations())


def sre_profile_passes(psi, n_x: int, **kw) -> dict:
    """Per-pass CUDA-event timing of the family transform launch sequence."""
    p, N = _psi_ptr(psi)
    ms = (ctypes.c_double * 4)()
    by = (ctypes.c_double * 4)()
    npass = ctypes.c_int(0)
    fpl = ctypes.c_longlong(0)
    _check(load().sre_profile_passes(p, N, n_x, ctypes.byref(_opts(**kw)), _stream(), ms, by,
                                     ctypes.byref(npass), ctypes.byref(fpl)))
    k = npass.value
    return {"n_passes": k, "ms": list(ms)[:k], "bytes": list(by)[:k], "families_per_launch": fpl.value}


def sre_pass_timing(enable: bool) -> dict:
    """Start (True) or stop (False) per-pass event timing inside sre_mc;
    returns the counters accumulated so far."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_longlong * 4)()
    by = (ctypes.c_double * 4)()
    _check(load().sre_pass_timing(1 if enable else 0, ms, n, by))
    return {"ms_sum": list(ms), "launches": list(n), "bytes_per_launch": list(by)}


def sre_exact_noalloc(psi, allow_nullity_error=False, **kw) -> dict:
    """sre_exact on the library's fixed scratch: allocates no device memory
    (N <= 13). For callers that cannot allocate at call time."""
    p, N = _psi_ptr(psi)
    r = Result()
    st = load().sre_exact_noalloc(p, N, ctypes.byref(_opts(**kw)), _stream(), ctypes.byref(r))
    _check(st, allow=(SRE_ENULLITY,) if allow_nullity_error else ())
    d = r.as_dict()
    d["status"] = st
    return d
