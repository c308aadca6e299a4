// k_tc.cuh -- the split-BF16 tensor-core form of the tile transform.
//
// A round over 4 bits of the tile is the matrix product Y = H_16 X with
// H_16[i][k] = (-1)^{popcount(i & k)} (the Kronecker power of (sqrt2 H) over
// the 4 bits, Eq. Z-FWHT's iteration) and X the 16 x (2^(M-4)) matrix of the
// tile's points along those bits (columns: every value of the other bits, real
// and imaginary parts separately). H_16's entries are exact in BF16; X is
// split into NSPLIT BF16 parts (x = hi + mid + lo, each the BF16 rounding of
// the remainder) and the NSPLIT products accumulate in FP32 on the tensor
// cores (mma.sync m16n8k16, BF16 x BF16 -> FP32). Remaining bits (fewer than
// 4) use the FP32 butterfly. The tile lives in shared memory (padded layout
// of TileCfg) between rounds.
#pragma once

#include <cuda_bf16.h>
#include "sre_internal.cuh"

namespace sre {

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    __nv_bfloat162 v;
    v.x = lo;
    v.y = hi;
    return *reinterpret_cast<uint32_t *>(&v);
}

// x = sum of NSPLIT BF16 parts (part 0 the largest)
template <int NSPLIT>
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 (&p)[NSPLIT]) {
    float r = x;
#pragma unroll
    for (int s = 0; s < NSPLIT; ++s) {
        p[s] = __float2bfloat16_rn(r);
        r = r - __bfloat162float(p[s]);
    }
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ __nv_bfloat16 hsign(int i, int k) {
    return __float2bfloat16_rn((__popc(i & k) & 1) ? -1.0f : 1.0f);
}

// A fragment of H_16 for this lane (m16n8k16, row-major A).
__device__ __forceinline__ void h16_fragment(uint32_t (&a)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    a[0] = pack_bf16x2(hsign(g, 2 * q), hsign(g, 2 * q + 1));
    a[1] = pack_bf16x2(hsign(g + 8, 2 * q), hsign(g + 8, 2 * q + 1));
    a[2] = pack_bf16x2(hsign(g, 2 * q + 8), hsign(g, 2 * q + 9));
    a[3] = pack_bf16x2(hsign(g + 8, 2 * q + 8), hsign(g + 8, 2 * q + 9));
}

// element index with the 4 bits p inserted at bit b of the column index c
__device__ __forceinline__ uint32_t ins4(uint32_t c, int b, uint32_t p) {
    return ((c >> b) << (b + 4)) | (p << b) | (c & ((1u << b) - 1u));
}

// One tensor-core round over bits [b, b+4) of the group's tile in shared
// memory; warps of the group take 8-column blocks in turn. In place: a warp
// reads and writes the same 16 x 8 block.
template <class Cfg, int NSPLIT>
__device__ __forceinline__ void tc_round(float2 *tile, int b, const uint32_t (&a)[4], int warp, int nwarps) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    constexpr int COLS = 1 << (Cfg::M - 4);
    for (int c0 = warp * 8; c0 < COLS; c0 += nwarps * 8) {
        const uint32_t cin = (uint32_t)(c0 + g);
        float2 xv[4];
        const uint32_t pin[4] = {(uint32_t)(2 * q), (uint32_t)(2 * q + 1), (uint32_t)(2 * q + 8), (uint32_t)(2 * q + 9)};
#pragma unroll
        for (int i = 0; i < 4; ++i) xv[i] = tile[Cfg::pad(ins4(cin, b, pin[i]))];
        float dre[4] = {0.f, 0.f, 0.f, 0.f}, dim[4] = {0.f, 0.f, 0.f, 0.f};
        __nv_bfloat16 pr[4][NSPLIT], pi[4][NSPLIT];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            split_bf16<NSPLIT>(xv[i].x, pr[i]);
            split_bf16<NSPLIT>(xv[i].y, pi[i]);
        }
#pragma unroll
        for (int s = NSPLIT - 1; s >= 0; --s) {   // smallest parts first
            mma_bf16_16816(dre, a, pack_bf16x2(pr[0][s], pr[1][s]), pack_bf16x2(pr[2][s], pr[3][s]));
            mma_bf16_16816(dim, a, pack_bf16x2(pi[0][s], pi[1][s]), pack_bf16x2(pi[2][s], pi[3][s]));
        }
        __syncwarp();
        // D(m, n): rows m = g, g+8 (output point), columns n = 2q, 2q+1
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t pout = (uint32_t)(g + ((i >> 1) << 3));
            const uint32_t cout = (uint32_t)(c0 + 2 * q + (i & 1));
            tile[Cfg::pad(ins4(cout, b, pout))] = make_float2(dre[i], dim[i]);
        }
        __syncwarp();
    }
}

// FP32 butterflies over bits [b, b+k) (k < 4) of the group's tile in shared
// memory: each thread of the group takes whole 2^k-point sub-vectors.
template <class Cfg>
__device__ __forceinline__ void simt_round_smem(float2 *tile, int b, int k, uint32_t t) {
    const int n_sub = 1 << (Cfg::M - k);
    for (int sidx = t; sidx < n_sub; sidx += Cfg::T) {
        const uint32_t base = ((uint32_t)(sidx >> b) << (b + k)) | ((uint32_t)sidx & ((1u << b) - 1u));
        float2 v[8];
        const int L = 1 << k;
        for (int p = 0; p < L; ++p) v[p] = tile[Cfg::pad(base | ((uint32_t)p << b))];
        for (int h = 1; h < L; h <<= 1)
            for (int p = 0; p < L; ++p)
                if (!(p & h)) {
                    const float2 u = v[p], w = v[p | h];
                    v[p] = make_float2(u.x + w.x, u.y + w.y);
                    v[p | h] = make_float2(u.x - w.x, u.y - w.y);
                }
        for (int p = 0; p < L; ++p) tile[Cfg::pad(base | ((uint32_t)p << b))] = v[p];
    }
}

// Tensor-core tile transform over bits [LO, M): registers (first mapping) ->
// shared memory -> rounds -> registers (last mapping). Requires one group per
// CTA or groups of whole warps.
template <class Cfg, int NSPLIT>
__device__ __forceinline__ void tc_tile_transform(float2 (&v)[Cfg::E], float2 *sm, uint32_t t, uint32_t grp) {
    float2 *tile = sm + grp * (uint32_t)Cfg::PSIZE;
    constexpr int A0 = Maps<Cfg>::first;
    constexpr int AL = Maps<Cfg>::last;
    {
        float2 *pb = tile + Cfg::pad(Cfg::elem(t, 0, A0));
#pragma unroll
        for (int k = 0; k < Cfg::E; ++k) pb[Cfg::pad((uint32_t)k << A0)] = v[k];
    }
    __syncthreads();
    uint32_t a[4];
    h16_fragment(a);
    constexpr int WPG = Cfg::T >= 32 ? Cfg::T / 32 : 1;   // warps per group
    const int warp = (int)(t >> 5);
    int b = Cfg::LO;
    static_assert(Cfg::T >= 32, "tensor-core rounds need whole warps per tile");
    for (; b + 4 <= Cfg::M; b += 4) {
        tc_round<Cfg, NSPLIT>(tile, b, a, warp, WPG);
        __syncthreads();
    }
    if (b < Cfg::M) {
        simt_round_smem<Cfg>(tile, b, Cfg::M - b, t);
        __syncthreads();
    }
    {
        const float2 *pb = tile + Cfg::pad(Cfg::elem(t, 0, AL));
#pragma unroll
        for (int k = 0; k < Cfg::E; ++k) v[k] = pb[Cfg::pad((uint32_t)k << AL)];
    }
}

} // namespace sre
