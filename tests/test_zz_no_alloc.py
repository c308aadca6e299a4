"""The allocation-free exact sweep (sre_exact_noalloc) against sre_exact.

sre_exact_noalloc serves callers that cannot allocate device memory at call
time (a device memory pool owned by another allocator, a fixed memory budget,
or no room for the synchronisation an allocation can bring). It runs the same
sweep on a scratch array the library reserves statically, so it must give the
same M_1..M_3 and nullity as sre_exact, on consecutive calls that reuse the
scratch, and must refuse sizes beyond the scratch before touching the device.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

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


def _call_abi(sre, psi):
    """The new entry point, called through the C ABI directly."""
    L = sre.load()
    N = psi.numel().bit_length() - 1
    r = sre.Result()
    o = sre.sre_default_opts()
    st = L.sre_exact_noalloc(ctypes.c_void_p(psi.data_ptr()), N, ctypes.byref(o),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(r))
    return st, r.as_dict()


def _states():
    g1 = inputs.random_clifford_tdoped_gates(10, 60, 4, 31)
    p1 = torch.zeros(1 << 10, dtype=torch.complex64, device="cuda")
    p1[0] = 1
    return [p1, g1, torch.from_numpy(inputs.haar_state(13, 5)).cuda(),
            torch.from_numpy(inputs.t_product_state(7, 3)).cuda()]


def test_noalloc_matches_sre_exact_on_consecutive_calls(sre):
    p1, g1, p2, p3 = _states()
    sre.apply_clifford_tdoped_circuit(p1, g1)
    for psi in (p1, p2, p3, p1):          # consecutive calls share the scratch
        st, r = _call_abi(sre, psi)
        ref = sre.sre_exact(psi, allow_nullity_error=True)
        assert st == ref["status"]
        assert np.max(np.abs(np.array(r["M"]) - np.array(ref["M"]))) < TOL_M
        assert r["nullity"] == ref["nullity"] and r["stab_count"] == ref["stab_count"]
        assert abs(r["parseval"] - ref["parseval"]) < 1e-9


def test_noalloc_binding_same_name(sre):
    psi = torch.from_numpy(inputs.t_product_state(9, 4)).cuda()
    a = sre.sre_exact_noalloc(psi)
    b = sre.sre_exact_noalloc(psi)
    ref = sre.sre_exact(psi)
    for r in (a, b):
        assert np.max(np.abs(np.array(r["M"]) - np.array(ref["M"]))) < TOL_M
        assert r["nullity"] == ref["nullity"] == 4


def test_noalloc_rejects_sizes_beyond_the_scratch(sre):
    psi = torch.zeros(1 << 14, dtype=torch.complex64, device="cuda")
    psi[0] = 1
    st, _ = _call_abi(sre, psi)
    assert st == sre.SRE_EINVAL
    assert "scratch" in sre.sre_last_error()


def test_noalloc_makes_no_device_allocation(sre):
    """The defining property: with the library's own workspace released, two
    calls of sre_exact_noalloc leave the library's allocation counter where it
    was (sre_exact without a workspace, by contrast, allocates again)."""
    psi = torch.from_numpy(inputs.haar_state(12, 7)).cuda()
    torch.cuda.synchronize()
    sre.sre_release_workspace()
    a0 = sre.sre_device_allocations()
    for _ in range(2):
        st, r = _call_abi(sre, psi)
        assert st == sre.SRE_OK
    assert sre.sre_device_allocations() == a0
    sre.sre_exact(psi)
    assert sre.sre_device_allocations() >= a0 + 1
