// k_tc05.cu -- tensor-map creation and the tcgen05 self-test GEMM.
//
// The self-test multiplies BF16 matrices with FP32 accumulation in TMEM:
// D[M x N] = A[M x K] B[N x K]^T (both operands K-major), one 128 x BN tile
// per CTA, K in blocks of 64, 32 or 16 (128-, 64- or 32-byte swizzle)
// brought in by TMA through a two-stage ring, K = 16 MMAs issued by one
// thread, then the
// accumulator read back by the four warps (warp w: rows 32 w .. 32 w + 31).
// It checks the descriptor and TMEM conventions the library's tensor-core
// kernels rely on against a plain matrix product.
#include <cudaTypedefs.h>
#include <mutex>

#include "k_tc05.cuh"
#include "sre_internal.cuh"

namespace sre {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
cudaError_t g_encode_err = cudaSuccess;
}

cudaError_t tc05_make_map_bf16(CUtensorMap *map, const void *base, unsigned long long rows, unsigned long long cols,
                               unsigned long long pitch_elems, unsigned box_rows, int sw, unsigned long long planes) {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        g_encode_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (g_encode_err == cudaSuccess && (q != cudaDriverEntryPointSuccess || !fn)) g_encode_err = cudaErrorNotSupported;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (g_encode_err != cudaSuccess) return g_encode_err;
    const unsigned box_cols = (unsigned)sw / 2;
    if ((sw != 128 && sw != 64 && sw != 32) || ((uintptr_t)base & 15) || (pitch_elems * 2) % 16 || cols % box_cols ||
        box_rows == 0 || box_rows > 256 || planes == 0)
        return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {cols, rows, planes};
    const cuuint64_t strides[2] = {pitch_elems * 2, pitch_elems * 2 * rows};
    const cuuint32_t box[3] = {box_cols, box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, planes > 1 ? 3 : 2, const_cast<void *>(base), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          sw == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                    : (sw == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B),
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, int SW>
__global__ void __launch_bounds__(128, 1) tc05_gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                           const __grid_constant__ CUtensorMap tb, float *D, int N,
                                                           int K, int *err) {
    using namespace tc05;
    constexpr int KB = SW / 2, KSTEPS = SW / 32;      // K per block, K = 16 MMA steps per block
    constexpr uint32_t ABYTES = 128 * SW, BBYTES = BN * SW, STAGE = ABYTES + BBYTES;
    constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
    extern __shared__ unsigned char smraw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + 2 * STAGE);
    uint64_t *done = full + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 2);
    int *last = reinterpret_cast<int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * BN;
    if (warp == 0) {
        tmem_alloc(tslot, TCOLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        mbar_init(full, 1);
        mbar_init(full + 1, 1);
        mbar_init(done, 1);
        mbar_init(done + 1, 1);
        fence_barrier_init();
        prefetch_tmap(&ta);
        prefetch_tmap(&tb);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    const int nk = K / KB;
    if (threadIdx.x == 0) {
        const long long deadline = clock64() + (1LL << 31);
        const uint32_t idesc = idesc_bf16_f32(128, BN);
        int committed = -1;
        bool ok = true;
        mbar_expect_tx(full, STAGE);
        tma_load_2d(base, &ta, 0, m0, full);
        tma_load_2d(base + ABYTES, &tb, 0, n0, full);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb & 1;
            unsigned char *sa = base + s * STAGE;
            if (!mbar_wait(full + s, (uint32_t)((kb >> 1) & 1), deadline)) { ok = false; break; }
            fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < KSTEPS; ++ks)
                mma_bf16(tmem, smem_desc<SW>(smem_u32(sa) + 32 * ks), smem_desc<SW>(smem_u32(sa + ABYTES) + 32 * ks),
                         idesc, (kb > 0 || ks > 0) ? 1u : 0u);
            mma_commit(done + s);
            committed = kb;
            if (kb + 1 < nk) {
                const int s1 = (kb + 1) & 1;
                if (kb >= 1 && !mbar_wait(done + s1, (uint32_t)(((kb - 1) >> 1) & 1), deadline)) { ok = false; break; }
                unsigned char *sb = base + s1 * STAGE;
                mbar_expect_tx(full + s1, STAGE);
                tma_load_2d(sb, &ta, (kb + 1) * KB, m0, full + s1);
                tma_load_2d(sb + ABYTES, &tb, (kb + 1) * KB, n0, full + s1);
            }
        }
        if (!ok) atomicOr(err, SRE_ERR_TIMEOUT);
        *last = committed;
    }
    __syncthreads();
    const int lk = *last;
    bool have = false;
    if (lk >= 0) have = mbar_wait(done + (lk & 1), (uint32_t)((lk >> 1) & 1), clock64() + (1LL << 31));
    if (lk >= 0 && !have && lane == 0) atomicOr(err, SRE_ERR_TIMEOUT);
    fence_after_sync();
    if (lk == nk - 1 && have) {
        const int row = m0 + 32 * warp + lane;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
            float *out = D + (size_t)row * N + n0 + c;
#pragma unroll
            for (int i = 0; i < 32; ++i) out[i] = v[i];
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

template <int SW>
cudaError_t launch_tc05_gemm_sw(const void *A, const void *B, float *D, int M, int N, int K, int *err,
                                cudaStream_t st) {
    constexpr int BN = 128;
    CUtensorMap ta, tb;
    cudaError_t e = tc05_make_map_bf16(&ta, A, (unsigned long long)M, (unsigned long long)K, (unsigned long long)K, 128, SW);
    if (e != cudaSuccess) return e;
    e = tc05_make_map_bf16(&tb, B, (unsigned long long)N, (unsigned long long)K, (unsigned long long)K, BN, SW);
    if (e != cudaSuccess) return e;
    const size_t smem = 1024 + 2 * (128 * SW + BN * SW) + 64;
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(tc05_gemm_kernel<BN, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    tc05_gemm_kernel<BN, SW><<<dim3(N / BN, M / 128), 128, smem, st>>>(ta, tb, D, N, K, err);
    return cudaGetLastError();
}

// swizzle: 128, 64 or 32 (bytes per operand row in shared memory)
cudaError_t launch_tc05_gemm_selftest(const void *A, const void *B, float *D, int M, int N, int K, int swizzle,
                                      int *err, cudaStream_t st) {
    if (M % 128 || N % 128 || K % 64 || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
    if (swizzle == 128) return launch_tc05_gemm_sw<128>(A, B, D, M, N, K, err, st);
    if (swizzle == 64) return launch_tc05_gemm_sw<64>(A, B, D, M, N, K, err, st);
    if (swizzle == 32) return launch_tc05_gemm_sw<32>(A, B, D, M, N, K, err, st);
    return cudaErrorInvalidValue;
}

} // namespace sre
