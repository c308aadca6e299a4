"""GPU: the fifth-generation tensor-core path (tcgen05.mma with TMEM
accumulators, TMA-loaded 128-byte-swizzled operands) against plain matrix
products. BF16 products are exact in FP32, so the only error is the FP32
accumulation over K: |dD| <= K 2^-23 max|a||b| is allowed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sre():
    import paper_2601_00761_gb300 as s
    from paper_2601_00761_gb300 import build
    build.build()
    s.load()
    return s


def _ref(A, B):
    return A.double().cpu().numpy() @ B.double().cpu().numpy().T


@pytest.mark.parametrize("swizzle", [128, 64, 32])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 256), (128, 256, 1024), (384, 128, 192)])
def test_gemm_random(sre, M, N, K, swizzle):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    D = sre.sre_tc_gemm_selftest(A, B, swizzle).double().cpu().numpy()
    ref = _ref(A, B)
    bound = K * 2.0**-23 * float(A.float().abs().max() * B.float().abs().max())
    assert np.max(np.abs(D - ref)) <= bound


@pytest.mark.parametrize("swizzle", [128, 64, 32])
def test_gemm_layout_is_exact_on_permutations(sre, swizzle):
    """A = a row permutation of the identity: D must be B's rows permuted,
    exactly (every product is one nonzero term)."""
    M = N = K = 256
    perm = torch.randperm(M, generator=torch.Generator().manual_seed(5))
    A = torch.zeros(M, K)
    A[torch.arange(M), perm] = 1.0
    B = torch.randn(N, K, generator=torch.Generator().manual_seed(6)).to(torch.bfloat16)
    D = sre.sre_tc_gemm_selftest(A.to(torch.bfloat16).cuda(), B.cuda(), swizzle).cpu()
    assert torch.equal(D, B.float().T[perm])


def test_gemm_hadamard_factor(sre):
    """X times the Sylvester matrix H_64 (entries +-1, exact in BF16): each
    row of D is the Walsh-Hadamard transform of a row of X over 64 points."""
    H = np.array([[(-1) ** bin(i & j).count("1") for j in range(64)] for i in range(64)], dtype=np.float32)
    X = torch.randn(128, 64, generator=torch.Generator().manual_seed(9)).to(torch.bfloat16)
    Hb = torch.from_numpy(np.tile(H, (2, 1))).to(torch.bfloat16)      # N = 128: H twice
    D = sre.sre_tc_gemm_selftest(X.cuda(), Hb.cuda()).double().cpu().numpy()
    want = X.double().numpy() @ H.T.astype(np.float64)
    assert np.max(np.abs(D[:, :64] - want)) < 64 * 2.0**-23 * float(X.float().abs().max())
    assert np.array_equal(D[:, :64], D[:, 64:])
