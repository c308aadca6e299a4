// k_tc05.cuh -- fifth-generation tensor-core (tcgen05) building blocks for
// sm_100-family parts: tensor-memory (TMEM) allocation, the shared-memory
// matrix and instruction descriptors of tcgen05.mma kind::f16, MMA issue and
// commit, TMEM loads, tensor-map (TMA) loads into shared memory and bounded
// mbarrier waits. All of it is inline PTX written from the PTX ISA.
//
// Layout used throughout: K-major BF16 operand tiles of 64 elements (128 B)
// per row, filled by TMA with the 128-byte swizzle, 8-row groups 1024 B
// apart; a tile's base is 1024-byte aligned. An MMA step of K = 16 reads
// 32 B of every row, so the k-th step of a 64-wide block starts 32 k bytes
// into the block.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sre {
namespace tc05 {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ------------------------------------------------------------- mbarriers
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait (one thread) for the completion of phase `parity`; false once the SM
// clock passes `deadline` without it.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long deadline) {
    while (!mbar_test(bar, parity)) {
        if (clock64() > deadline) return false;
    }
    return true;
}

// ------------------------------------------------------------------ TMA
// 2-D tiled load of the box at (c0 = inner element, c1 = row) of `map` into
// shared memory, completing on `bar` (which expects the bytes).
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)map) : "memory");
}

// ------------------------------------------------------------------ TMEM
// Allocate `ncols` (a power of two, 32..512) TMEM columns; the whole warp
// calls it; the address lands in *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ----------------------------------------------------------- descriptors
// Shared-memory matrix descriptor of a K-major tile whose rows are SW bytes
// (SW = 128, 64 or 32) swizzled as TMA's SW-byte mode writes them: start address,
// leading-dimension byte offset (unused for swizzled K-major tiles), stride
// between 8-row groups (8 SW bytes), both in 16-byte units, the fixed version
// bits 46..48 = 0b001, base offset 0, and the layout type in bits 61..63
// (2 = 128-byte swizzle, 4 = 64-byte, 6 = 32-byte).
template <int SW>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    static_assert(SW == 128 || SW == 64 || SW == 32, "128-, 64- or 32-byte swizzle");
    const uint64_t start = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    const uint64_t lbo = 1;
    const uint64_t sbo = (8 * SW) >> 4;
    const uint64_t layout = SW == 128 ? 2 : (SW == 64 ? 4 : 6);
    return start | (lbo << 16) | (sbo << 32) | (1ull << 46) | (layout << 61);
}
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) { return smem_desc<128>(saddr); }

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// BF16 A and B (bits 7-9, 10-12 = 1), optional negation of A (bit 13),
// K-major A and B (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N, bool neg_a = false) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on `bar` once every tcgen05 operation this thread issued so far has
// completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w of a
// warpgroup reads lanes 32 (w % 4) .. + 31).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

} // namespace tc05

// Host: a tensor map over row-major BF16 matrices (planes x rows x cols, cols
// contiguous, row pitch `pitch_elems`, plane pitch rows * pitch_elems) with
// boxes of sw/2 columns x box_rows rows x 1 plane and the sw-byte swizzle
// (sw = 128, 64 or 32). planes = 1 gives a 2-D map. Returns cudaSuccess or an
// error.
cudaError_t tc05_make_map_bf16(CUtensorMap *map, const void *base, unsigned long long rows, unsigned long long cols,
                               unsigned long long pitch_elems, unsigned box_rows, int sw = 128,
                               unsigned long long planes = 1);

} // namespace sre
