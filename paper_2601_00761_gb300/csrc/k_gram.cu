// k_gram.cu -- the Gram matrix C = Psi Psi^H of a bipartite state on the
// tensor cores (SM, mixed states: the reduced state of the first N_A qubits
// is rho_A = C, C[a][a'] = sum_e psi(a, e) conj psi(a', e), and the partial
// transform reads h_{x_A}(a) = C[a][a ^ x_A]).
//
// Psi is the complex64 state viewed as d_A x d_B (row a = the low N_A bits,
// column e = the rest; element (a, e) at psi[a + d_A e]). With X = Re Psi and
// Y = Im Psi, C = (X X^T + Y Y^T) + i (Y X^T - X Y^T): four real products
// with K = d_B. Every FP32 value is split into three BF16 parts (x = x0 + x1 +
// x2 exactly up to the last bits of x2) and a product x y is taken as the six
// part products x_p y_q with p + q <= 2, which leaves an error of about
// 2^-24 |x y|, the FP32 rounding level.
//
// 1. gram_split_kernel transposes Psi into six K-major BF16 planes
//    P[c * 3 + p][a][e] (c = 0: X, 1: Y; p the part).
// 2. gram_tc_kernel: one 128 x 128 tile (I, J) of C per CTA, I <= J only;
//    K in blocks of 16 (32-byte rows, TMA with the 32-byte swizzle), a
//    four-stage ring of 12 contiguous 4 KB boxes per block (X_I, Y_I, X_J,
//    Y_J, three parts each); one thread issues the TMA loads and the 24 MMAs
//    per block into a fresh TMEM accumulator (D_re, D_im), alternating
//    between two; eight warps add each block's accumulator into FP32
//    register sums and write the tile and, off the diagonal, its conjugate
//    transpose. With several chunks of K the tile is added to C.
// 3. gram_diag_kernel: the diagonal (the trace of rho_A and the x_A = 0
//    family) summed in FP64 and written over the tiles' diagonal.
// 4. gram_simt_kernel: small shapes (d_A < 128 or d_B < 32), FP32 products
//    summed in FP64 per entry.
#include "k_tc05.cuh"
#include "sre_internal.cuh"
#include "k_fp64.cuh"

#include <cuda_bf16.h>

namespace sre {

// ------------------------------------------------------------ split
// Planes: 6 x (d_A x dBc) BF16, tiled so that every 128-row x 16-column block
// the Gram kernel loads is 4 KB of contiguous memory: element (a, e) of a
// plane at ((a / 128) * (dBc / 16) + e / 16) * 2048 + (a % 128) * 16 + e % 16.
// This chunk covers columns e0 .. e0 + dBc of Psi.
__global__ void __launch_bounds__(256) gram_split_kernel(const float2 *psi, int NA, long long e0, int dBc_log2,
                                                         __nv_bfloat16 *planes) {
    __shared__ float2 t[32][33];
    const unsigned long long dA = 1ULL << NA, dBc = 1ULL << dBc_log2;
    const unsigned long long a0 = (unsigned long long)blockIdx.x * 32, c0 = (unsigned long long)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    // read 32 rows a (contiguous) x 32 columns e
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int col = ty + 8 * k;
        t[col][tx] = psi[(a0 + tx) + dA * (unsigned long long)(e0 + (long long)(c0 + col))];
    }
    __syncthreads();
    const size_t plane = (size_t)dA * dBc;
    const unsigned long long neb = dBc / 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int row = ty + 8 * k;                    // a = a0 + row, e = c0 + tx
        const float2 v = t[tx][row];
        const unsigned long long a = a0 + row, e = c0 + tx;
        const size_t o = ((a >> 7) * neb + (e >> 4)) * 2048 + (a & 127) * 16 + (e & 15);
        const float xs[2] = {v.x, v.y};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float x = xs[c];
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            const float r1 = x - __bfloat162float(h);
            const __nv_bfloat16 m = __float2bfloat16_rn(r1);
            const float r2 = r1 - __bfloat162float(m);
            const __nv_bfloat16 l = __float2bfloat16_rn(r2);
            planes[(size_t)(3 * c + 0) * plane + o] = h;
            planes[(size_t)(3 * c + 1) * plane + o] = m;
            planes[(size_t)(3 * c + 2) * plane + o] = l;
        }
    }
}

// ------------------------------------------------------------ tensor cores
constexpr int GRAM_T = 128;                    // tile rows / columns
constexpr int GRAM_KB = 16;                    // K per block (32-byte rows, one MMA step)
constexpr uint32_t GRAM_BOX = GRAM_T * 32;     // bytes of one 128 x 16 BF16 box (contiguous)
constexpr uint32_t GRAM_STAGE = 12 * GRAM_BOX; // X_I, Y_I, X_J, Y_J x 3 parts
constexpr int GRAM_NS = 4;                     // stages in the ring
constexpr int GRAM_EPI = 256;                  // epilogue threads (8 warps)
constexpr int GRAM_THREADS = GRAM_EPI + 32;    // + one warp issuing TMA and MMA
constexpr size_t GRAM_SMEM = 1024 + GRAM_NS * (size_t)GRAM_STAGE + 256;
// K blocks accumulated in one TMEM buffer before the epilogue warps drain it
#ifndef SRE_GRAM_R
#define SRE_GRAM_R 1
#endif
constexpr int GRAM_R = SRE_GRAM_R;

// tile index -> (I, J) with I <= J over nt x nt tiles (row-major upper triangle)
__device__ __forceinline__ void tri_tile(int idx, int nt, int &I, int &J) {
    int i = 0, rem = idx;
    while (rem >= nt - i) { rem -= nt - i; ++i; }
    I = i;
    J = i + rem;
}

// The tensor cores' FP32 accumulation is not rounded to nearest: summed over
// a long K in one accumulator, coherent terms (a diagonal-dominant or pure
// rho_A) lose about 2^-24 of the sum per addition. Each K block therefore
// starts a fresh accumulator in one of two TMEM buffers (columns 0..255 and
// 256..511: D_re, D_im), and the epilogue warps add it, while the next block
// runs, into FP32 register sums (round to nearest): 24 tensor-core additions
// per block instead of 24 per block times the number of blocks.
//
// Warp 8 (lane 0) loads the stages by TMA and issues the MMAs; warps 0..7
// drain the TMEM buffers (warp w reads lanes 32 (w % 4) .. + 31, columns
// 64 (w / 4) .. + 63 of D_re and D_im) and write the tile at the end.
__global__ void __launch_bounds__(GRAM_THREADS, 1) gram_tc_kernel(const __grid_constant__ CUtensorMap tp, float2 *C,
                                                                  int NA, int dBc_log2, int accumulate_c, int *err) {
    using namespace tc05;
    extern __shared__ unsigned char smraw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + GRAM_NS * GRAM_STAGE);   // [NS] stage loaded
    uint64_t *sfree = full + GRAM_NS;                                           // [NS] stage read by the MMAs
    uint64_t *tready = sfree + GRAM_NS;                                         // [2] TMEM buffer holds a block
    uint64_t *tfree = tready + 2;                                               // [2] TMEM buffer drained
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tfree + 2);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long dA = 1ULL << NA;
    const int nt = (int)(dA / GRAM_T);
    int I, J;
    tri_tile((int)blockIdx.x, nt, I, J);
    const int r0I = I * GRAM_T, r0J = J * GRAM_T;
    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    if (threadIdx.x == GRAM_EPI) {
        for (int i = 0; i < GRAM_NS; ++i) {
            mbar_init(full + i, 1);
            mbar_init(sfree + i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tready + i, 1);
            mbar_init(tfree + i, GRAM_EPI);
        }
        *abort_flag = 0;
        fence_barrier_init();
        prefetch_tmap(&tp);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    const int nk = (1 << dBc_log2) / GRAM_KB;
    const long long deadline = clock64() + (1LL << 32);
    if (warp == GRAM_EPI / 32) {
        if (lane == 0) {
            const uint32_t id_pos = idesc_bf16_f32(GRAM_T, GRAM_T, false);
            const uint32_t id_neg = idesc_bf16_f32(GRAM_T, GRAM_T, true);
            // block (row block rb, K block kb) of a plane starts at row (rb * nk + kb) * 128 of the map
            auto load_stage = [&](int kb, int s) {
                unsigned char *st = base + s * GRAM_STAGE;
                mbar_expect_tx(full + s, GRAM_STAGE);
                // slot (m, p): m = 0 X_I, 1 Y_I, 2 X_J, 3 Y_J; plane = 3 (m & 1) + p
#pragma unroll
                for (int m = 0; m < 4; ++m)
#pragma unroll
                    for (int p = 0; p < 3; ++p)
                        tma_load_3d(st + (m * 3 + p) * GRAM_BOX, &tp, 0, ((m < 2 ? I : J) * nk + kb) * GRAM_T,
                                    3 * (m & 1) + p, full + s);
            };
            bool ok = true;
            for (int kb = 0; kb < nk && kb < GRAM_NS; ++kb) load_stage(kb, kb);
            for (int kb = 0; kb < nk && ok; ++kb) {
                // K block kb goes into TMEM buffer b of accumulation group gi
                const int s = kb % GRAM_NS, gi = kb / GRAM_R, pos = kb - gi * GRAM_R, b = gi & 1;
                if (!mbar_wait(full + s, (uint32_t)((kb / GRAM_NS) & 1), deadline)) { ok = false; break; }
                if (pos == 0 && gi >= 2 && !mbar_wait(tfree + b, (uint32_t)(((gi - 2) >> 1) & 1), deadline)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t sb = smem_u32(base + s * GRAM_STAGE);
                const uint32_t dre = tmem + 256u * (uint32_t)b, dim = dre + 128u;
                auto slot = [&](int m, int p) { return smem_desc<32>(sb + (m * 3 + p) * GRAM_BOX); };
                // part pairs (p, q) with p + q <= 2, smallest first
                const int PP[6] = {1, 2, 0, 1, 0, 0}, QQ[6] = {1, 0, 2, 0, 1, 0};
#pragma unroll
                for (int u = 0; u < 6; ++u) {
                    const int p = PP[u], q = QQ[u];
                    const uint32_t acc = (u > 0 || pos > 0) ? 1u : 0u;
                    mma_bf16(dre, slot(0, p), slot(2, q), id_pos, acc);     // X_I X_J^T
                    mma_bf16(dre, slot(1, p), slot(3, q), id_pos, 1u);      // + Y_I Y_J^T
                    mma_bf16(dim, slot(1, p), slot(2, q), id_pos, acc);     // Y_I X_J^T
                    mma_bf16(dim, slot(0, p), slot(3, q), id_neg, 1u);      // - X_I Y_J^T
                }
                mma_commit(sfree + s);
                if (pos == GRAM_R - 1 || kb == nk - 1) mma_commit(tready + b);
                // refill the stage of the previous block (its MMAs ran while this block's were queued)
                if (kb >= 1 && kb - 1 + GRAM_NS < nk) {
                    const int sp = (kb - 1) % GRAM_NS;
                    if (!mbar_wait(sfree + sp, (uint32_t)(((kb - 1) / GRAM_NS) & 1), deadline)) { ok = false; break; }
                    load_stage(kb - 1 + GRAM_NS, sp);
                }
            }
            if (!ok) {
                atomicOr(err, SRE_ERR_TIMEOUT);
                atomicExch(abort_flag, 1);
            }
        }
    } else {
        // epilogue warps: FP32 running sums of 64 columns of D_re and D_im
        float sre_[64], sim_[64];
#pragma unroll
        for (int k = 0; k < 64; ++k) { sre_[k] = 0.f; sim_[k] = 0.f; }
        const uint32_t lrow = (uint32_t)(32 * (warp & 3)) << 16;
        const uint32_t c0 = 64u * (uint32_t)(warp >> 2);
        bool ok = true;
        const int ng = (nk + GRAM_R - 1) / GRAM_R;
        for (int g = 0; g < ng; ++g) {
            const int s = g & 1;
            bool ready = false;
            while (!(ready = mbar_test(tready + s, (uint32_t)((g >> 1) & 1)))) {
                if (clock64() > deadline || *(volatile int *)abort_flag) break;
            }
            if (!__all_sync(0xffffffffu, ready)) { ok = false; break; }
            fence_after_sync();
            const uint32_t b = tmem + lrow + 256u * (uint32_t)s + c0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[32];
                tmem_ld32(b + 32u * h, v);
#pragma unroll
                for (int k = 0; k < 32; ++k) sre_[32 * h + k] += v[k];
                tmem_ld32(b + 128u + 32u * h, v);
#pragma unroll
                for (int k = 0; k < 32; ++k) sim_[32 * h + k] += v[k];
            }
            fence_before_sync();
            mbar_arrive(tfree + s);
        }
        if (!ok && lane == 0) atomicOr(err, SRE_ERR_TIMEOUT);
        if (ok) {
            const unsigned long long i = (unsigned long long)r0I + 32 * (warp & 3) + lane;
#pragma unroll
            for (int k = 0; k < 64; ++k) {
                const unsigned long long jj = (unsigned long long)r0J + c0 + k;
                float2 v = make_float2(sre_[k], sim_[k]);
                float2 *pc = C + i + dA * jj;
                if (accumulate_c) { const float2 o = *pc; v.x += o.x; v.y += o.y; }
                *pc = v;
            }
            if (I != J) {
                // C[j][i] = conj C[i][j]: 64 consecutive j of this thread's row i
                float2 *row = C + (unsigned long long)r0J + c0 + dA * i;
#pragma unroll
                for (int k = 0; k < 64; k += 2) {
                    float4 w = make_float4(sre_[k], -sim_[k], sre_[k + 1], -sim_[k + 1]);
                    float4 *pr = reinterpret_cast<float4 *>(row + k);
                    if (accumulate_c) {
                        const float4 o = *pr;
                        w.x += o.x; w.y += o.y; w.z += o.z; w.w += o.w;
                    }
                    *pr = w;
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------ small shapes
__global__ void __launch_bounds__(256) gram_simt_kernel(const float2 *psi, int NA, int NB, float2 *C) {
    const unsigned long long dA = 1ULL << NA, dB = 1ULL << NB;
    const unsigned long long idx = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= dA * dA) return;
    const unsigned long long i = idx % dA, j = idx / dA;     // C[i][j] at i + dA j
    double re = 0.0, im = 0.0;
    for (unsigned long long e = 0; e < dB; ++e) {
        const float2 a = psi[i + dA * e], b = psi[j + dA * e];
        // a conj(b)
        re += (double)(a.x * b.x + a.y * b.y);
        im += (double)(a.y * b.x - a.x * b.y);
    }
    C[i + dA * j] = make_float2((float)re, (float)im);
}

// Diagonal of C, sum_e |psi(a, e)|^2, in FP64 (written over the tensor-core
// tile's diagonal). It holds the trace of rho_A and every c_{0,z}, which
// dominate the moments of a strongly mixed rho_A; the tensor cores' FP32
// accumulation leaves them about 1e-6 off, summed in FP64 they carry only
// the final FP32 rounding.
constexpr int GRAM_DIAG_WARPS = 32;
__global__ void __launch_bounds__(32 * GRAM_DIAG_WARPS) gram_diag_kernel(const float2 *psi, int NA, int NB, float2 *C) {
    // one block per 32 consecutive a (coalesced 256-byte rows of Psi); warp
    // w sums e = w, w + 32, ... (exact FP64 squares, widened in integer
    // operations); the partial sums are added in a fixed order, so the result
    // does not depend on scheduling
    __shared__ double part[GRAM_DIAG_WARPS][32];
    const unsigned long long dA = 1ULL << NA, dB = 1ULL << NB;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned long long a = (unsigned long long)blockIdx.x * 32 + lane;
    double acc = 0.0;
    if (a < dA) {
#pragma unroll 4
        for (unsigned long long e = (unsigned long long)w; e < dB; e += GRAM_DIAG_WARPS) {
            const float2 v = psi[a + dA * e];
            const double vx = f2d(v.x), vy = f2d(v.y);
            acc = fma(vx, vx, acc);
            acc = fma(vy, vy, acc);
        }
    }
    part[w][lane] = acc;
    __syncthreads();
    if (w == 0 && a < dA) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < GRAM_DIAG_WARPS; ++i) t += part[i][lane];
        C[a + dA * a] = make_float2((float)t, 0.0f);
    }
}

// K chunk (columns of Psi per split) bounded so the planes stay within 2^27 elements each
int gram_chunk_log2(int N, int NA) {
    const int nb = N - NA;
    const int cap = 27 - NA;
    return nb < cap ? nb : (cap < 5 ? 5 : cap);
}

size_t gram_plane_bytes(int N, int NA) {
    if (NA < 7 || N - NA < 5) return 0;
    return (size_t)6 * ((size_t)1 << NA) * ((size_t)1 << gram_chunk_log2(N, NA)) * sizeof(__nv_bfloat16);
}

cudaError_t launch_gram(const float2 *psi, int N, int NA, float2 *C, void *planes, int *err, int *launches,
                        cudaStream_t st) {
    const int NB = N - NA;
    *launches = 0;
    if (NA < 7 || NB < 5) {
        const unsigned long long n = 1ULL << (2 * NA);
        gram_simt_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(psi, NA, NB, C);
        *launches = 1;
        return cudaGetLastError();
    }
    const int cl = gram_chunk_log2(N, NA);
    const unsigned long long dA = 1ULL << NA, dBc = 1ULL << cl;
    const int nt = (int)(dA / GRAM_T);
    const int ntiles = nt * (nt + 1) / 2;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRAM_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap tp;
    // each plane as (d_A dBc / 16) rows of 16 columns (the tiled layout of gram_split_kernel)
    cudaError_t e = tc05_make_map_bf16(&tp, planes, dA * (dBc / GRAM_KB), GRAM_KB, GRAM_KB, GRAM_T, 32, 6);
    if (e != cudaSuccess) return e;
    for (long long e0 = 0; e0 < (1LL << NB); e0 += (long long)dBc) {
        gram_split_kernel<<<dim3((unsigned)(dA / 32), (unsigned)(dBc / 32)), 256, 0, st>>>(
            psi, NA, e0, cl, reinterpret_cast<__nv_bfloat16 *>(planes));
        gram_tc_kernel<<<ntiles, GRAM_THREADS, GRAM_SMEM, st>>>(tp, C, NA, cl, e0 > 0 ? 1 : 0, err);
        *launches += 2;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    gram_diag_kernel<<<(unsigned)((dA + 31) / 32), 32 * GRAM_DIAG_WARPS, 0, st>>>(psi, NA, NB, C);
    *launches += 1;
    return cudaGetLastError();
}

} // namespace sre
