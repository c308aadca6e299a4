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
                                                          unsigned long long *zs, float *cz) {
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
    const long long gf = a.fam_base + slot;
    const uint32_t t = threadIdx.x;

    const int N = a.N, n = a.n;
    const unsigned long long x = a.xs[gf] & ((1ULL << N) - 1ULL);
    const int j = x ? 63 - __clzll((long long)x) : n;
    const unsigned long long half = 1ULL << n;
    const DrawInfo dr = draws[(size_t)gf * z_per_x + kdraw];
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
    const size_t out = (size_t)gf * z_per_x + kdraw;
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
                       cudaStream_t st) {
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
    zsample_kernel<Cfg, SRC, PREC><<<grid, Cfg::NT, smem, st>>>(a, draws, z_per_x, zs, cz);
    return cudaGetLastError();
}

template <class Cfg, int SRC>
cudaError_t launch_zs(const PassArgs &a, const DrawInfo *draws, int z_per_x, unsigned long long *zs, float *cz,
                      cudaStream_t st) {
    if (a.precision == 0 || Cfg::T < 32) return launch_zs1<Cfg, SRC, 0>(a, draws, z_per_x, zs, cz, st);
    if constexpr (Cfg::T >= 32) {
        if (a.precision == 2) return launch_zs1<Cfg, SRC, 2>(a, draws, z_per_x, zs, cz, st);
        if (a.precision == 3) return launch_zs1<Cfg, SRC, 3>(a, draws, z_per_x, zs, cz, st);
    }
    return cudaErrorInvalidValue;
}

template <int M> using SampleSingle = TileCfg<float, M, 0, (M < 5 ? M : 5), 1>;

cudaError_t launch_zsample(int single, int M, const PassArgs &a, const DrawInfo *draws, int z_per_x,
                           unsigned long long *zs, float *cz, cudaStream_t st) {
    if (single) {
        switch (M) {
#define C(m) case m: return launch_zs<SampleSingle<m>, SRC_PSI_FAMILY>(a, draws, z_per_x, zs, cz, st);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13) C(14)
#undef C
        default: return cudaErrorInvalidValue;
        }
    }
    switch (M) {
#define C(m) case m: return launch_zs<TileCfg<float, m, 0, 5, 1>, SRC_BUF>(a, draws, z_per_x, zs, cz, st);
    C(10) C(11) C(12) C(13) C(14)
#undef C
    default: return cudaErrorInvalidValue;
    }
}

} // namespace sre
