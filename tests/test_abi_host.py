"""CPU tests of the C ABI: the library loads, exports every entry point that
include/sre.h declares, and its host-side logic (plans, workspace sizes,
argument checks) behaves -- none of these calls touches a GPU."""
import ctypes
import os
import re

import pytest

import paper_2601_00761_gb300 as sre

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2601_00761_gb300 import build
    build.build()
    return sre.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "sre.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"SRE_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("sre_exact", "sre_mc", "pauli_x_marginal", "stabilizer_nullity",
                 "apply_clifford_tdoped_circuit", "sre_exact_batched", "sre_family_spectrum"):
        assert want in names


def test_every_declared_symbol_is_exported(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_binding_exposes_the_same_names(L):
    for name in _declared():
        assert callable(getattr(sre, name)), name


def test_version(L):
    assert "sm_103a" in sre.sre_version()


@pytest.mark.parametrize("N,passes,bits", [
    (1, 1, [0]), (10, 1, [9]), (15, 1, [14]), (16, 2, [2, 13]), (18, 2, [4, 13]),
    (24, 2, [10, 13]), (25, 3, [5, 6, 13]), (30, 3, [8, 8, 13])])
def test_plans(L, N, passes, bits):
    p = sre.sre_make_plan(N)
    assert p["n_passes"] == passes
    assert p["pass_bits"] == bits
    assert sum(p["pass_bits"]) == N - 1
    # passes tile the bit range [0, N-1) top-down without gaps
    top = N - 1
    for lo, k in zip(p["pass_lo"], p["pass_bits"]):
        assert lo + k == top
        top = lo
    assert top == 0


def test_batched_argument_errors_do_not_touch_the_gpu(L):
    r = (sre.Result * 2)()
    o = sre.sre_default_opts()
    ptrs = (ctypes.c_void_p * 2)(0x1000, 0x2000)
    ns = (ctypes.c_int * 2)(10, 12)
    assert L.sre_exact_batched(ptrs, ns, 0, ctypes.byref(o), None, 0, None, r) == sre.SRE_OK      # empty batch
    assert L.sre_exact_batched(ptrs, ns, -1, ctypes.byref(o), None, 0, None, r) == sre.SRE_EINVAL
    assert L.sre_exact_batched(None, ns, 2, ctypes.byref(o), None, 0, None, r) == sre.SRE_EINVAL
    assert L.sre_exact_batched(ptrs, ns, 2, ctypes.byref(o), None, 0, None, None) == sre.SRE_EINVAL
    big = (ctypes.c_int * 2)(10, 21)                                                          # N in 1..20
    assert L.sre_exact_batched(ptrs, big, 2, ctypes.byref(o), None, 0, None, r) == sre.SRE_EINVAL
    odd = (ctypes.c_void_p * 2)(0x1000, 0x2004)                                               # 8-byte aligned psi
    assert L.sre_exact_batched(odd, ns, 2, ctypes.byref(o), None, 0, None, r) == sre.SRE_EINVAL
    assert L.sre_exact_batched(ptrs, ns, 2, ctypes.byref(o), _fake_ptr(0x3000), 1 << 20, None, r) == sre.SRE_ENOTSUP
    q = sre.Opts(0, 1e-6, 0, 0, 0, 3)
    assert L.sre_exact_batched(ptrs, ns, 2, ctypes.byref(q), None, 0, None, r) == sre.SRE_EINVAL


def test_autotune_clear_arguments(L):
    assert L.sre_autotune_clear(33) == sre.SRE_EINVAL
    assert L.sre_autotune_clear(-1) == sre.SRE_EINVAL
    assert L.sre_autotune_clear(0) == sre.SRE_OK
    assert L.sre_autotune_clear(18) == sre.SRE_OK


def test_plan_options(L):
    p = sre.sre_make_plan(24, radix_log2=11, tile_log2=6)
    assert p["pass_bits"] == [6, 6, 11]
    assert sre.sre_make_plan(24, radix_log2=13, tile_log2=10)["pass_bits"] == [10, 13]
    # the bottom strided pass keeps its columns below its row stride
    p = sre.sre_make_plan(18, radix_log2=10, tile_log2=4)
    assert p["pass_bits"] == [3, 4, 10]
    p = sre.sre_make_plan(16, radix_log2=10, tile_log2=2)
    assert p["pass_bits"] == [2, 3, 10]
    assert sre.sre_make_plan(24, x_batch=3)["x_batch"] == 3
    # batches stay within 8 GiB of FP32 intermediate, except that states of
    # N >= 29 still take 8 families per launch within 32 GiB
    assert sre.sre_make_plan(24)["x_batch"] == 128
    assert sre.sre_make_plan(28)["x_batch"] == 8
    assert sre.sre_make_plan(30)["x_batch"] == 8
    assert sre.sre_make_plan(31)["x_batch"] == 4
    assert sre.sre_make_plan(32)["x_batch"] == 2


def test_workspace_sizes(L):
    a = sre.sre_workspace_bytes(18, -1)
    b = sre.sre_workspace_bytes(18, -1, x_batch=8)
    assert a > b > 0
    m = sre.sre_workspace_bytes(24, sre.SRE_MC_MARGINAL, 4096, 256)
    u = sre.sre_workspace_bytes(24, sre.SRE_MC_UNIFORM, 4096, 1)
    assert m > u > 0
    # the marginal needs at least p(x) + its FP64 work buffer and one intermediate
    assert m > 2 * 8 * 2**24 + 8 * 2**23


def _fake_ptr(addr):
    return ctypes.c_void_p(addr)


def test_argument_errors_do_not_touch_the_gpu(L):
    r = sre.Result()
    o = sre.sre_default_opts()
    assert L.sre_exact(None, 10, ctypes.byref(o), None, 0, None, ctypes.byref(r)) == sre.SRE_EINVAL
    assert "NULL" in sre.sre_last_error()
    assert L.sre_exact(_fake_ptr(0x1001), 10, ctypes.byref(o), None, 0, None, ctypes.byref(r)) == sre.SRE_EINVAL
    assert "aligned" in sre.sre_last_error()
    assert L.sre_exact(_fake_ptr(0x1000), 0, ctypes.byref(o), None, 0, None, ctypes.byref(r)) == sre.SRE_EINVAL
    assert L.sre_exact(_fake_ptr(0x1000), 27, ctypes.byref(o), None, 0, None, ctypes.byref(r)) == sre.SRE_EINVAL
    assert L.sre_mc(_fake_ptr(0x1000), 10, 7, 10, 1, 0, 0, None, None, 0, None, ctypes.byref(r),
                    None, None, None) == sre.SRE_EINVAL
    assert L.sre_mc(_fake_ptr(0x1000), 10, 1, 1, 1, 0, 0, None, None, 0, None, ctypes.byref(r),
                    None, None, None) == sre.SRE_EINVAL
    assert L.sre_mc(_fake_ptr(0x1000), 10, 1, 10, 0, 0, 0, None, None, 0, None, ctypes.byref(r),
                    None, None, None) == sre.SRE_EINVAL
    bad = sre.Opts(9, 1e-6, 0, 0, 0)
    assert L.sre_exact(_fake_ptr(0x1000), 10, ctypes.byref(bad), None, 0, None, ctypes.byref(r)) == sre.SRE_EINVAL
    neg = sre.Opts(0, 1e-6, 0, 0, -1)
    assert L.sre_exact(_fake_ptr(0x1000), 10, ctypes.byref(neg), None, 0, None, ctypes.byref(r)) == sre.SRE_EINVAL
    queue = sre.Opts(0, 1e-6, 0, 0, 0, 2)     # batch_queue is 0 or 1
    assert L.sre_exact(_fake_ptr(0x1000), 10, ctypes.byref(queue), None, 0, None, ctypes.byref(r)) == sre.SRE_EINVAL
    for eps in (0.5, 2.0, float("nan")):     # nullity tolerance outside (0, 0.5)
        wide = sre.Opts(0, eps, 0, 0, 0)
        assert L.sre_exact(_fake_ptr(0x1000), 10, ctypes.byref(wide), None, 0, None, ctypes.byref(r)) == sre.SRE_EINVAL
        nu, cnt = ctypes.c_int(), ctypes.c_longlong()
        assert L.stabilizer_nullity(_fake_ptr(0x1000), 10, ctypes.c_double(eps), ctypes.byref(nu), ctypes.byref(cnt),
                                    None) == sre.SRE_EINVAL
    g = (sre.Gate * 1)(sre.Gate(9, 0, 0))
    assert L.apply_clifford_tdoped_circuit(_fake_ptr(0x1000), 4, g, 1, None) == sre.SRE_EINVAL
    g = (sre.Gate * 1)(sre.Gate(3, 1, 1))
    assert L.apply_clifford_tdoped_circuit(_fake_ptr(0x1000), 4, g, 1, None) == sre.SRE_EINVAL
    g = (sre.Gate * 1)(sre.Gate(0, 4, 0))
    assert L.apply_clifford_tdoped_circuit(_fake_ptr(0x1000), 4, g, 1, None) == sre.SRE_EINVAL
    mats = (ctypes.c_float * 32)()
    for bad in ((1, 1), (0, 4), (-1, 2)):
        pr = (ctypes.c_int * 2)(*bad)
        assert L.apply_two_qubit_gates(_fake_ptr(0x1000), 4, mats, pr, 1, None) == sre.SRE_EINVAL
    assert L.apply_two_qubit_gates(_fake_ptr(0x1000), 1, mats, (ctypes.c_int * 2)(0, 1), 1, None) == sre.SRE_EINVAL
    assert L.apply_two_qubit_gates(_fake_ptr(0x1000), 4, None, None, 1, None) == sre.SRE_EINVAL
    assert L.sre_family_spectrum(_fake_ptr(0x1000), 4, 16, None, _fake_ptr(0x2000), None) == sre.SRE_EINVAL
    assert L.pauli_x_marginal(_fake_ptr(0x1000), 4, None, None, 0, None) == sre.SRE_EINVAL
    p = sre.Plan()
    assert L.sre_make_plan(33, None, ctypes.byref(p)) == sre.SRE_EINVAL
    mr = sre.MixedResult()
    for N, NA in ((8, 0), (8, 9), (20, 16), (31, 4)):
        assert L.sre_mixed(_fake_ptr(0x1000), N, NA, None, 0, None, ctypes.byref(mr)) == sre.SRE_EINVAL
    assert L.sre_mixed(_fake_ptr(0x1000), 8, 4, _fake_ptr(0x1000), 16, None, ctypes.byref(mr)) == sre.SRE_EINVAL
    assert "workspace" in sre.sre_last_error()
    assert L.sre_workspace_bytes(10, 5, 10, 1, None, ctypes.byref(ctypes.c_size_t())) == sre.SRE_EINVAL


def test_mixed_workspace_bytes(L):
    # the d_A x d_A complex64 Gram matrix and the six BF16 split planes of Psi
    # (d_A x d_B each) that the tensor-core Gram kernel reads
    want = 8 * 4 ** 10 + 6 * 2 * 2 ** 20
    assert want < sre.sre_mixed_workspace_bytes(20, 10) < want + (1 << 20)
    # small subsystems take the SIMT route and no planes
    assert sre.sre_mixed_workspace_bytes(12, 6) < 8 * 4 ** 6 + (1 << 20)


def test_structs_match_header_layout():
    # sre_gate is a packed 3-byte row; sre_opts / sre_result field order as declared
    assert ctypes.sizeof(sre.Gate) == 3
    assert sre.Opts.eps_null.offset == 8 and sre.Opts.batch_queue.offset == 28 and ctypes.sizeof(sre.Opts) == 32
    assert sre.Result.M.offset == 0 and sre.Result.parseval.offset == 15 * 8
    assert sre.Result.stab_count.offset == 16 * 8
    assert sre.Result.r2.offset == 22 * 8 and ctypes.sizeof(sre.Result) == 23 * 8


def test_oracle_not_imported_by_the_package():
    import sys
    import subprocess
    code = ("import sys; import paper_2601_00761_gb300 as s; s.load(); "
            "assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules), 'oracle imported'")
    subprocess.check_call([sys.executable, "-c", code], cwd=ROOT)
    pkg = os.path.join(ROOT, "paper_2601_00761_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "sre_oracle" not in txt, f
