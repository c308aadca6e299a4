// k_sample.cu -- the second level of the z sampler.
//
// A draw has already picked a z-range r (2^RL consecutive z in natural order)
// and the remainder t' of its target inside that range. The range is the
// output of one last-pass tile: the kernel recomputes that tile with the same
// prologue, rounds and c-pair code as the fused moments epilogue (so every
// c^2 is bit-identical to the one that entered the range weight), lays the
// range's c^2 out in z order in shared memory and returns the smallest z with
// C(z) > t', C the running sum over the range of the c^2 in u32 fixed point
// (2^31 quanta per range weight) -- exact, so every association agrees.
#include "k_misc.cuh"
#include "k_pass.cuh"

namespace sre {

template <class Cfg, int SRC, int PREC>
__global__ void __launch_bounds__(Cfg::NT) zsample_kernel(const PassArgs a, const DrawInfo *draws, int z_per_x,
                                                          unsigned long long *zs, float *cz,
                                                          const unsigned long long *perm) {
    typedef float R;
    typedef float2 C2;
    static_assert(Cfg::G == 1, "one tile per CTA");
    extern __shared__ __align__(16) unsigned char smraw[];
    C2 *sm = reinterpret_cast<C2 *>(smraw);
    double *seg = reinterpret_cast<double *>(smraw + sizeof(C2) * (size_t)Cfg::PSIZE);

    const long long idx = (long long)blockIdx.x + 65535LL * (long long)blockIdx.y;
    if (idx >= a.n_fam * (long long)z_per_x) return;   // uniform over the CTA
    const long long slot = idx / z_per_x;
    const int kdraw = (int)(idx - slot * z_per_x);
    const long long gf = a.fam_base + slot;                          // processing order
    const long long of = perm ? (long long)perm[gf] : gf;           // the family's own index
    const uint32_t t = threadIdx.x;

    const int N = a.N, n = a.n;
    const unsigned long long x = a.xs[gf] & ((1ULL << N) - 1ULL);
    const int j = x ? 63 - __clzll((long long)x) : n;
    const unsigned long long half = 1ULL << n;
    const DrawInfo dr = draws[(size_t)of * z_per_x + kdraw];
    const int RL = Cfg::M;
    const unsigned long long zstart = dr.range << RL;
    const unsigned long long zp0 = ((zstart >> (j + 1)) << j) | (zstart & ((1ULL << j) - 1ULL));
    const unsigned long long tile = zp0 >> Cfg::M;
    const unsigned long long gbase = tile << Cfg::M;

    // The per-draw FP64 scalars (fixed-point scale, target in quanta, s) are
    // formed once by thread 0 and passed through shared memory: the FP64
    // pipe is narrow on this part and a divide in every thread would
    // dominate the kernel. The barrier after the transform orders the write.
    constexpr int NW = (Cfg::NT + 31) / 32;
    unsigned long long *bc = reinterpret_cast<unsigned long long *>(seg) + NW + 1;
    if (t == 0) {
        const double scale = dr.wr > 0.0 ? 0x1.0p31 / dr.wr : 0.0;
        double tq = dr.t * scale;
        if (tq < 0.0) tq = 0.0;
        bc[0] = tq < 1.8e19 ? (unsigned long long)tq : ~0ULL;
        float *bf = reinterpret_cast<float *>(bc + 1);
        bf[0] = (float)scale;
        bf[1] = (float)(*a.s_ptr);
    }

    C2 v[Cfg::E];
    pass_prologue<Cfg, SRC>(v, a, a.psi, slot, x, j, half, gbase, t);
    if constexpr (PREC == 0) tile_transform<Cfg>(v, sm, t, 0);
    else tc_tile_transform<Cfg, PREC>(v, sm, t, 0);
    __syncthreads();

    // The range's c^2 in z order as u32 fixed-point quanta (scale 2^31 per
    // range weight) and its signed c; one padding word per 32 entries keeps
    // each thread's 32 consecutive entries conflict-free. Integer prefix sums
    // are exact in any association, so the thread segments tile the range
    // exactly and every target has one owner.
    uint32_t *wq = reinterpret_cast<uint32_t *>(smraw);
    float *cv = reinterpret_cast<float *>(wq + (1 << RL) + ((1 << RL) >> 5));
    auto pp = [](uint32_t p) { return p + (p >> 5); };
    const float scf = reinterpret_cast<const float *>(bc + 1)[0];
    const R s = reinterpret_cast<const float *>(bc + 1)[1];
    const unsigned long long T = bc[0];
    constexpr int AL = Maps<Cfg>::last;
#pragma unroll
    for (int k = 0; k < Cfg::E; ++k) {
        unsigned long long z0, z1;
        R c0, c1;
        family_pair<R, C2>(x, j, s, v[k], gbase | Cfg::elem(t, k, AL), z0, z1, c0, c1);
        if ((z0 >> RL) == dr.range) {
            const uint32_t q = pp((uint32_t)(z0 - zstart));
            wq[q] = __float2uint_rn(fminf(c0 * c0 * scf, 4.0e9f));
            cv[q] = c0;
        }
        if ((z1 >> RL) == dr.range) {
            const uint32_t q = pp((uint32_t)(z1 - zstart));
            wq[q] = __float2uint_rn(fminf(c1 * c1 * scf, 4.0e9f));
            cv[q] = c1;
        }
    }
    __syncthreads();

    constexpr int PER = (1 << Cfg::M) / Cfg::NT;
    const int lo = t * PER;
    unsigned long long own = 0;
    for (int i = 0; i < PER; ++i) own += wq[pp(lo + i)];
    // warps of the CTA (the smallest tiles have fewer than 32 threads)
    constexpr int WL = Cfg::NT < 32 ? Cfg::NT : 32;
    constexpr unsigned MASK = Cfg::NT < 32 ? ((1u << Cfg::NT) - 1u) : 0xffffffffu;
    unsigned long long incl = own;
#pragma unroll
    for (int o = 1; o < WL; o <<= 1) {
        const unsigned long long up = __shfl_up_sync(MASK, incl, o);
        if ((int)(threadIdx.x & 31) >= o) incl += up;
    }
    unsigned long long *wsum = reinterpret_cast<unsigned long long *>(seg);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == WL - 1) wsum[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int q = 0; q < NW; ++q) { const unsigned long long v0 = wsum[q]; wsum[q] = run; run += v0; }
        wsum[NW] = run;
    }
    __syncthreads();
    const unsigned long long before = wsum[wid] + incl - own;
    const unsigned long long total = wsum[NW];
    const size_t out = (size_t)of * z_per_x + kdraw;
    if (T < total && before <= T && T < before + own) {
        unsigned long long run = before;
        int pick = lo + PER - 1;
        for (int i = 0; i < PER; ++i) {
            run += wq[pp(lo + i)];
            if (run > T) { pick = lo + i; break; }
        }
        zs[out] = zstart + (unsigned long long)pick;
        cz[out] = cv[pp(pick)];
    } else if (threadIdx.x == 0 && !(T < total)) {
        int pick = (1 << RL) - 1;
        while (pick > 0 && wq[pp(pick)] == 0u) --pick;
        zs[out] = zstart + (unsigned long long)pick;
        cz[out] = cv[pp(pick)];
    }
}

template <class Cfg, int SRC, int PREC>
cudaError_t launch_zs1(const PassArgs &a, const DrawInfo *draws, int z_per_x, unsigned long long *zs, float *cz,
                       const unsigned long long *perm, cudaStream_t st) {
    const size_t smem = sizeof(float2) * (size_t)Cfg::PSIZE + sizeof(double) * ((Cfg::NT + 31) / 32 + 4);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(zsample_kernel<Cfg, SRC, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long nd = a.n_fam * (long long)z_per_x;
    dim3 grid((unsigned)(nd < 65535 ? nd : 65535), (unsigned)((nd + 65534) / 65535));
    zsample_kernel<Cfg, SRC, PREC><<<grid, Cfg::NT, smem, st>>>(a, draws, z_per_x, zs, cz, perm);
    return cudaGetLastError();
}

template <class Cfg, int SRC>
cudaError_t launch_zs(const PassArgs &a, const DrawInfo *draws, int z_per_x, unsigned long long *zs, float *cz,
                      const unsigned long long *perm, cudaStream_t st) {
    if (a.precision == 0 || Cfg::T < 32) return launch_zs1<Cfg, SRC, 0>(a, draws, z_per_x, zs, cz, perm, st);
    if constexpr (Cfg::T >= 32) {
        if (a.precision == 2) return launch_zs1<Cfg, SRC, 2>(a, draws, z_per_x, zs, cz, perm, st);
        if (a.precision == 3) return launch_zs1<Cfg, SRC, 3>(a, draws, z_per_x, zs, cz, perm, st);
    }
    return cudaErrorInvalidValue;
}

// Fine ranges (multi-pass plans whose last tiles exceed 2^ZR_FINE points):
// one warp per draw. The draw's range is 2^ZR_FINE consecutive z, and every
// z' = z with bit j removed that it needs lies in one aligned block of
// 2^ZR_FINE outputs of a last-pass tile. The Walsh transform factorises over
// disjoint bit sets, so that block is the ZR_FINE-bit transform of the tile's
// input summed over its M - ZR_FINE top bits with signs (-1)^{F.h}, F the
// block's top bits: the warp reads the tile once, folds it, and transforms
// 2^ZR_FINE points instead of 2^M.
constexpr int FOLD_WARPS = 4;   // three CTAs per SM

// shared-memory points per warp: the two-stage ring of 2^RL-point blocks
// (the transpose and the fixed-point range reuse it afterwards)
constexpr int FOLD_WSTRIDE = 2 * (1 << ZR_FINE);
constexpr size_t FOLD_SMEM = sizeof(float2) * (size_t)FOLD_WARPS * FOLD_WSTRIDE + sizeof(uint64_t) * 2 * FOLD_WARPS;
__device__ __forceinline__ uint64_t *fold_bars(unsigned char *smraw) {
    return reinterpret_cast<uint64_t *>(smraw + sizeof(float2) * (size_t)FOLD_WARPS * FOLD_WSTRIDE);
}

// mbarrier and bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk)
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the asynchronous proxy
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// bytes (a multiple of 16) from global src to shared dst (both 16-byte
// aligned), completing on bar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Waiting budget of a warp: about 2^31 SM cycles (about a second) for all of
// its waits together, and one more such budget for draining its copies after a
// timeout, so a warp that meets a stuck copy returns within about two seconds.
constexpr long long WAIT_BUDGET = 1LL << 31;

// warp-uniform wait for the completion of phase `parity` of bar; false once
// the SM clock has passed `deadline` without it
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long deadline) {
    for (;;) {
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
        if (clock64() > deadline) return false;
    }
}

template <int M>
__global__ void __launch_bounds__(32 * FOLD_WARPS) zsample_fold_kernel(const PassArgs a, const DrawInfo *draws,
                                                                      int z_per_x, unsigned long long *zs,
                                                                      float *cz, const unsigned long long *perm) {
    constexpr int RL = ZR_FINE, NB = 1 << RL, H = 1 << (M - RL), SW = NB + NB / 32;
    static_assert(M > RL && RL == 10, "a warp holds 32 x 32 folded points");
    static_assert(FOLD_WSTRIDE >= SW, "the transpose and the range fit the warp's region");
    extern __shared__ __align__(16) unsigned char smraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *sm = reinterpret_cast<float2 *>(smraw) + warp * FOLD_WSTRIDE;
    const long long idx = (long long)blockIdx.x * FOLD_WARPS + warp;
    if (idx >= a.n_fam * (long long)z_per_x) return;      // uniform over the warp
    const long long slot = idx / z_per_x;
    const int kdraw = (int)(idx - slot * z_per_x);
    const long long gf = a.fam_base + slot;                          // processing order
    const long long of = perm ? (long long)perm[gf] : gf;           // the family's own index
    const int N = a.N, n = a.n;
    const unsigned long long x = a.xs[gf] & ((1ULL << N) - 1ULL);
    const int j = x ? 63 - __clzll((long long)x) : n;
    const size_t out = (size_t)of * z_per_x + kdraw;
    const DrawInfo dr = draws[out];
    const unsigned long long zstart = dr.range << RL;
    const unsigned long long zp0 = ((zstart >> (j + 1)) << j) | (zstart & ((1ULL << j) - 1ULL));
    const unsigned long long zblk = zp0 & ~(unsigned long long)(NB - 1);
    const unsigned long long tile = zblk >> M;
    const uint32_t F = (uint32_t)(zblk >> RL) & (uint32_t)(H - 1);
    const float2 *src = reinterpret_cast<const float2 *>(a.src) + (size_t)slot * (size_t)a.slot_elems +
                        (size_t)(tile << M) + lane;

    // fold: f[k] = sum_h (-1)^{F.h} y[h 2^RL + 32 k + lane]
    float2 f[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) f[k] = make_float2(0.f, 0.f);
    // The tile's 2^(M-RL) blocks of 2^RL points (8 KB each) arrive by bulk
    // asynchronous copies into a two-stage ring of the warp's shared memory,
    // each stage completing on its own mbarrier; lane 0 issues block h + 2
    // into a stage once the warp has folded block h out of it. Every wait is
    // bounded: past the bound the warp records a timeout in the error word,
    // waits (bounded again) for its copies still in flight and returns.
    {
        float2 *ring = sm;                                   // 2 x 2^RL points
        uint64_t *bar = fold_bars(smraw) + 2 * warp;
        const float2 *tsrc = src - lane;
        if (lane == 0) {
            mbar_init(bar, 1);
            mbar_init(bar + 1, 1);
            fence_mbar_init();
#pragma unroll
            for (int h = 0; h < 2 && h < H; ++h) {
                mbar_expect_tx(bar + h, NB * 8u);
                bulk_g2s(ring + h * NB, tsrc + (size_t)h * NB, NB * 8u, bar + h);
            }
        }
        __syncwarp();
        bool ok = true;
        const long long deadline = clock64() + WAIT_BUDGET;     // one budget for every wait of the warp
#pragma unroll 1
        for (int h = 0; h < H; ++h) {
            const int st = h & 1;
            if (!mbar_wait_bounded(bar + st, (uint32_t)((h >> 1) & 1), deadline)) {
                ok = false;
                // the copies still in flight (this stage's and, if issued, the
                // other's) share one more budget; a copy that has not landed
                // by then may still be writing the warp's shared memory when
                // the kernel returns, and the error word reports it
                const long long drain = clock64() + WAIT_BUDGET;
                for (int q = h; q < H && q < h + 2; ++q) mbar_wait_bounded(bar + (q & 1), (uint32_t)((q >> 1) & 1), drain);
                break;
            }
            const float sg = (__popc(F & (uint32_t)h) & 1) ? -1.f : 1.f;
            const float2 sg2 = make_float2(sg, sg);
            const float2 *sb = ring + st * NB + lane;
#pragma unroll
            for (int k = 0; k < 32; ++k) f[k] = fma2(sg2, sb[32 * k], f[k]);
            __syncwarp();
            if (lane == 0 && h + 2 < H) {
                mbar_expect_tx(bar + st, NB * 8u);
                bulk_g2s(ring + st * NB, tsrc + (size_t)(h + 2) * NB, NB * 8u, bar + st);
            }
        }
        if (!ok) {
            if (lane == 0 && a.err_flag) atomicOr(a.err_flag, SRE_ERR_TIMEOUT);
            return;
        }
        __syncwarp();
    }
    // ZR_FINE-bit transform: bits 5..9 in registers, then bits 0..4 after a
    // transpose through shared memory (padded: conflict-free both ways)
    butterflies<float2, 32, 0, 5>(f);
#pragma unroll
    for (int k = 0; k < 32; ++k) sm[33 * k + lane] = f[k];
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 32; ++k) f[k] = sm[33 * lane + k];
    __syncwarp();
    butterflies<float2, 32, 0, 5>(f);          // lane l, slot k: output 32 l + k

    // per-draw scalars once per warp (the FP64 pipe is narrow on this part)
    float s = 0.f, scf = 0.f;
    unsigned long long T = 0;
    if (lane == 0) {
        s = (float)(*a.s_ptr);
        const double scale = dr.wr > 0.0 ? 0x1.0p31 / dr.wr : 0.0;
        double tq = dr.t * scale;
        if (tq < 0.0) tq = 0.0;
        T = tq < 1.8e19 ? (unsigned long long)tq : ~0ULL;
        scf = (float)scale;
    }
    s = __shfl_sync(0xffffffffu, s, 0);
    scf = __shfl_sync(0xffffffffu, scf, 0);
    T = __shfl_sync(0xffffffffu, T, 0);

    // the range's c^2 in z order as u32 fixed-point quanta (2^31 per range
    // weight) and its signed c; lane l then owns entries 32 l .. 32 l + 31
    uint32_t *wq = reinterpret_cast<uint32_t *>(sm);
    float *cv = reinterpret_cast<float *>(wq + SW);
    auto pp = [](uint32_t p) { return p + (p >> 5); };
    // c(z0), c(z1) of z' = zblk + 32 lane + k as in the last pass's epilogue
    // (z < 2^31: 32-bit indices; z0 = z' with 0 inserted at bit j)
    const uint32_t x32 = (uint32_t)x, r32 = (uint32_t)dr.range, zs32 = (uint32_t)zstart;
    const uint32_t hm = ~((1u << j) - 1u), jb = 1u << j;
    const uint32_t zl = (uint32_t)zblk + 32u * (uint32_t)lane;
    const float sc = 2.0f * s;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const uint32_t zp = zl + (uint32_t)k;
        const uint32_t z0 = zp + (zp & hm), z1 = z0 | jb;
        float c0, c1;
        if (x) {
            const int k0 = __popc(x32 & z0);
            const float re = sc * f[k].x, im = sc * f[k].y;
            c0 = (float)sgn_phase(k0) * ((k0 & 1) ? im : re);
            c1 = (float)sgn_phase(k0 + 1) * ((k0 & 1) ? re : im);
        } else {
            c0 = s * (f[k].x + f[k].y);
            c1 = s * (f[k].x - f[k].y);
        }
        if ((z0 >> RL) == r32) {
            const uint32_t q = pp(z0 - zs32);
            wq[q] = __float2uint_rn(fminf(c0 * c0 * scf, 4.0e9f));
            cv[q] = c0;
        }
        if ((z1 >> RL) == r32) {
            const uint32_t q = pp(z1 - zs32);
            wq[q] = __float2uint_rn(fminf(c1 * c1 * scf, 4.0e9f));
            cv[q] = c1;
        }
    }
    __syncwarp();

    const uint32_t lo = 32u * (uint32_t)lane;
    unsigned long long own = 0;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) own += wq[pp(lo + i)];
    unsigned long long incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long up = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += up;
    }
    const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
    const unsigned long long before = incl - own;
    if (T < total) {
        if (before <= T && T < before + own) {     // exactly one lane
            unsigned long long run = before;
            uint32_t pick = lo + 31;
            for (int i = 0; i < 32; ++i) {
                run += wq[pp(lo + i)];
                if (run > T) { pick = lo + i; break; }
            }
            zs[out] = zstart + pick;
            cz[out] = cv[pp(pick)];
        }
    } else {
        // target at or beyond the fixed-point total (FP32 rounding of the
        // range weight): the last z of nonzero weight
        int last = -1;
        for (int i = 31; i >= 0; --i)
            if (wq[pp(lo + i)] != 0u) { last = (int)(lo + i); break; }
        const int m = __reduce_max_sync(0xffffffffu, last);
        if (lane == 0) {
            const uint32_t pick = m >= 0 ? (uint32_t)m : 0u;
            zs[out] = zstart + pick;
            cz[out] = cv[pp(pick)];
        }
    }
}

// One warp waits on an mbarrier whose expected bytes exceed the one 16-byte
// copy issued to it, so the phase never completes: the bounded wait must give
// up and record SRE_ERR_TIMEOUT (the copy itself has landed by then).
__global__ void __launch_bounds__(32) wait_selftest_kernel(const float4 *src, int *err) {
    __shared__ __align__(16) float4 buf[2];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar, 32u);
        bulk_g2s(buf, src, 16u, &bar);
    }
    __syncwarp();
    if (!mbar_wait_bounded(&bar, 0u, clock64() + WAIT_BUDGET) && threadIdx.x == 0) atomicOr(err, SRE_ERR_TIMEOUT);
}

cudaError_t launch_wait_selftest(const void *src16, int *err, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(reinterpret_cast<const float4 *>(src16), err);
    return cudaGetLastError();
}

template <int M>
cudaError_t launch_fold(const PassArgs &a, const DrawInfo *draws, int z_per_x, unsigned long long *zs, float *cz,
                        const unsigned long long *perm, cudaStream_t st) {
    constexpr size_t smem = FOLD_SMEM;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(zsample_fold_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long nd = a.n_fam * (long long)z_per_x;
    const long long nb = (nd + FOLD_WARPS - 1) / FOLD_WARPS;
    if (nb > 0x7fffffffLL) return cudaErrorInvalidValue;
    zsample_fold_kernel<M><<<(unsigned)nb, 32 * FOLD_WARPS, smem, st>>>(a, draws, z_per_x, zs, cz, perm);
    return cudaGetLastError();
}

template <int M> using SampleSingle = TileCfg<float, M, 0, (M < 5 ? M : 5), 1>;

cudaError_t launch_zsample(int single, int fine, int M, const PassArgs &a, const DrawInfo *draws, int z_per_x,
                           unsigned long long *zs, float *cz, const unsigned long long *perm, cudaStream_t st) {
    if (fine) {
        switch (M) {
        case 11: return launch_fold<11>(a, draws, z_per_x, zs, cz, perm, st);
        case 12: return launch_fold<12>(a, draws, z_per_x, zs, cz, perm, st);
        case 13: return launch_fold<13>(a, draws, z_per_x, zs, cz, perm, st);
        case 14: return launch_fold<14>(a, draws, z_per_x, zs, cz, perm, st);
        default: return cudaErrorInvalidValue;
        }
    }
    if (single) {
        switch (M) {
#define C(m) case m: return launch_zs<SampleSingle<m>, SRC_PSI_FAMILY>(a, draws, z_per_x, zs, cz, perm, st);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13) C(14)
#undef C
        default: return cudaErrorInvalidValue;
        }
    }
    switch (M) {
#define C(m) case m: return launch_zs<TileCfg<float, m, 0, 5, 1>, SRC_BUF>(a, draws, z_per_x, zs, cz, perm, st);
    C(10) C(11) C(12) C(13) C(14)
#undef C
    default: return cudaErrorInvalidValue;
    }
}

} // namespace sre
