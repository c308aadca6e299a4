// k_misc.cu -- normalisation, reductions, the FP64 CDF scan, Philox draws,
// the two-level z sampler and the MC statistics.
#include "k_misc.cuh"
#include "k_pass_dispatch.cuh"
#include "k_fp64.cuh"

namespace sre {

// ------------------------------------------------------------------ Philox
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (hi, lo) = M * c products with a Weyl key schedule.
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        const unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// Uniform of stream (seed), counter (ctr0 + i, lane, 0, 0): word 0, 53 bits.
__device__ __forceinline__ double mc_uniform(unsigned long long seed, unsigned long long ctr0,
                                             unsigned long long i, unsigned long long lane) {
    unsigned long long c[4] = {ctr0 + i, lane, 0ULL, 0ULL};
    philox4x64_10(c, seed, 0ULL);
    return (double)(c[0] >> 11) * 0x1.0p-53;
}

__global__ void philox_test_kernel(const unsigned long long *ctr_key, unsigned long long *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long c[4] = {ctr_key[6 * i], ctr_key[6 * i + 1], ctr_key[6 * i + 2], ctr_key[6 * i + 3]};
    philox4x64_10(c, ctr_key[6 * i + 4], ctr_key[6 * i + 5]);
    for (int w = 0; w < 4; ++w) out[4 * i + w] = c[w];
}

// ------------------------------------------------------------ reductions
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) s += red[w];
    return s;
}

// sum |psi|^2 in FP64: fixed grid, per-block partials
__global__ void __launch_bounds__(256) norm2_partial_kernel(const float2 *psi, unsigned long long d,
                                                            double *partial) {
    __shared__ double red[8];
    double acc = 0.0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; b < d; b += stride) {
        const float2 u = __ldg(psi + b);
        const double ux = f2d(u.x), uy = f2d(u.y);
        acc = fma(ux, ux, acc);
        acc = fma(uy, uy, acc);
    }
    acc = block_sum<256>(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) norm2_final_kernel(const double *partial, int np, double *scal) {
    __shared__ double red[8];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) acc += partial[i];
    acc = block_sum<256>(acc, red);
    if (threadIdx.x == 0) {
        scal[SCAL_NORM2] = acc;
        scal[SCAL_S] = acc > 0.0 ? 1.0 / acc : 0.0;
    }
}

cudaError_t launch_norm2(const float2 *psi, int N, double *scal, double *partial, cudaStream_t st) {
    const unsigned long long d = 1ULL << N;
    int nb = NORM_BLOCKS;
    if ((unsigned long long)nb * 256ULL > d) nb = (int)((d + 255) / 256);
    norm2_partial_kernel<<<nb, 256, 0, st>>>(psi, d, partial);
    norm2_final_kernel<<<1, 256, 0, st>>>(partial, nb, scal);
    return cudaGetLastError();
}

// tile partials -> family sums; z-range weights scattered to W[fam][range]
__global__ void __launch_bounds__(256) fam_reduce_kernel(const TilePartial *tp, long long n_fam, int tiles,
                                                         const unsigned long long *xs, long long fam_base,
                                                         int N, int M_last, int RL, FamMoments *fm,
                                                         long long fm_base, float *W, long long nr,
                                                         const unsigned long long *perm) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long f = (long long)blockIdx.x * 8 + warp;
    if (f >= n_fam) return;
    const int n = N - 1;
    unsigned long long x = xs ? xs[fam_base + f] : (unsigned long long)(fam_base + f);
    x &= (1ULL << N) - 1ULL;
    const int j = x ? 63 - __clzll((long long)x) : n;
    // plain FP64: a family's tile partials are FP32 sums (relative error about
    // 1e-7), far above this sum's rounding
    double m0 = 0, m1 = 0, m2 = 0, m3 = 0, c = 0;
    for (int t = lane; t < tiles; t += 32) {
        const TilePartial &p = tp[(size_t)f * tiles + t];
        m0 += p.m[0]; m1 += p.m[1]; m2 += p.m[2]; m3 += p.m[3]; c += (double)p.cand;
        if (W) {
            const unsigned long long zt = (unsigned long long)t << M_last;
            const unsigned long long rA = insert0(zt, j) >> RL;
            const unsigned long long rB = (j < RL) ? rA + 1 : rA + (1ULL << (j - RL));
            W[(size_t)f * nr + rA] = (float)p.w[0];
            W[(size_t)f * nr + rB] = (float)p.w[1];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m0 += __shfl_xor_sync(0xffffffffu, m0, o);
        m1 += __shfl_xor_sync(0xffffffffu, m1, o);
        m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        m3 += __shfl_xor_sync(0xffffffffu, m3, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        FamMoments &o = fm[perm ? (long long)perm[fam_base + f] : fm_base + f];
        o.m[0] = m0; o.m[1] = m1; o.m[2] = m2; o.m[3] = m3;
        o.cand = (unsigned long long)c;
    }
}

cudaError_t launch_fam_reduce(const TilePartial *tp, long long n_fam, int tiles, const unsigned long long *xs,
                              long long fam_base, int N, int M_last, int RL, FamMoments *fm, long long fm_base,
                              float *W, long long nr, cudaStream_t st, const unsigned long long *perm) {
    fam_reduce_kernel<<<(unsigned)((n_fam + 7) / 8), 256, 0, st>>>(tp, n_fam, tiles, xs, fam_base, N, M_last, RL,
                                                                  fm, fm_base, W, nr, perm);
    return cudaGetLastError();
}

// totals over families (exact sweep): per-block partials over contiguous
// chunks (fixed order), then one block; also the list of candidate families
// (order irrelevant: the FP64 counts are integers).
__global__ void __launch_bounds__(256) exact_partial_kernel(const FamMoments *fm, long long n_fam, double *partial,
                                                            unsigned long long *flag_list,
                                                            unsigned long long *n_flag) {
    __shared__ double red[8];
    const long long per = (n_fam + gridDim.x - 1) / gridDim.x;
    const long long lo = (long long)blockIdx.x * per, hi = lo + per < n_fam ? lo + per : n_fam;
    NeuSum s0, s1, s2, s3, sq;
    double c = 0;
    for (long long f = lo + threadIdx.x; f < hi; f += 256) {
        const FamMoments &m = fm[f];
        s0.add(m.m[0]); s1.add(m.m[1]); s2.add(m.m[2]); s3.add(m.m[3]); c += (double)m.cand;
        if (f > 0) sq.add(m.m[1] * m.m[1]);
        if (m.cand && flag_list) {
            unsigned long long pos = atomicAdd(n_flag, 1ULL);
            flag_list[pos] = (unsigned long long)f;
        }
    }
    double a0 = s0.value(), a1 = s1.value(), a2 = s2.value(), a3 = s3.value(), q = sq.value();
    a0 = block_sum<256>(a0, red);
    a1 = block_sum<256>(a1, red);
    a2 = block_sum<256>(a2, red);
    a3 = block_sum<256>(a3, red);
    c = block_sum<256>(c, red);
    q = block_sum<256>(q, red);
    if (threadIdx.x == 0) {
        double *o = partial + 6 * blockIdx.x;
        o[0] = a0; o[1] = a1; o[2] = a2; o[3] = a3; o[4] = c; o[5] = q;
    }
}

__global__ void __launch_bounds__(256) exact_final_kernel(const double *partial, int n_part, const FamMoments *fm0,
                                                          double *out) {
    __shared__ double red[8];
    for (int a = 0; a < 6; ++a) {
        NeuSum ns;
        for (int i = threadIdx.x; i < n_part; i += 256) ns.add(partial[6 * i + a]);
        const double s = block_sum<256>(ns.value(), red);
        if (threadIdx.x == 0) out[a] = s;
    }
    if (threadIdx.x == 0) out[6] = fm0[0].m[1];
}

cudaError_t launch_exact_totals(const FamMoments *fm, long long n_fam, double *partial, int n_part,
                                double *out, unsigned long long *flag_list, unsigned long long *n_flag,
                                cudaStream_t st) {
    exact_partial_kernel<<<n_part, 256, 0, st>>>(fm, n_fam, partial, flag_list, n_flag);
    exact_final_kernel<<<1, 256, 0, st>>>(partial, n_part, fm, out);
    return cudaGetLastError();
}

__global__ void sum_u64_kernel(const unsigned long long *v, long long n, unsigned long long *out) {
    __shared__ unsigned long long red[256];
    unsigned long long a = 0;
    for (long long i = threadIdx.x; i < n; i += 256) a += v[i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

cudaError_t launch_sum_u64(const unsigned long long *v, long long n, unsigned long long *out, cudaStream_t st) {
    sum_u64_kernel<<<1, 256, 0, st>>>(v, n, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------- CDF scan
// Inclusive FP64 scan in natural index order, fixed association (chunks of
// SCAN_CHUNK elements; 256 threads x 16 consecutive elements per chunk).
__global__ void __launch_bounds__(256) scan_chunk_sums(const double *p, unsigned long long n, double *bsum) {
    __shared__ double red[8];
    const unsigned long long base = (unsigned long long)blockIdx.x * SCAN_CHUNK + threadIdx.x * 16ULL;
    double a = 0.0;
#pragma unroll
    for (int i = 0; i < 16; ++i)
        if (base + i < n) a += p[base + i];
    // fixed-order block total: per-thread partials summed in thread order
    __shared__ double part[256];
    part[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < 256; ++t) s += part[t];
        bsum[blockIdx.x] = s;
    }
    (void)red;
}

__global__ void __launch_bounds__(256) scan_block_offsets(double *bsum, long long nb) {
    // exclusive prefix of bsum, in place, sequential over fixed segments
    __shared__ double seg[257];
    const long long per = (nb + 255) / 256;
    const long long lo = threadIdx.x * per, hi = lo + per < nb ? lo + per : nb;
    double s = 0.0;
    for (long long i = lo; i < hi; ++i) s += bsum[i];
    seg[threadIdx.x + 1] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        seg[0] = 0.0;
        for (int t = 1; t <= 256; ++t) seg[t] += seg[t - 1];
    }
    __syncthreads();
    double run = seg[threadIdx.x];
    for (long long i = lo; i < hi; ++i) {
        const double v = bsum[i];
        bsum[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(256) scan_chunk_apply(const double *p, unsigned long long n, const double *boff,
                                                        double *cdf) {
    __shared__ double part[257];
    const unsigned long long base = (unsigned long long)blockIdx.x * SCAN_CHUNK + threadIdx.x * 16ULL;
    double loc[16];
    double a = 0.0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        loc[i] = (base + i < n) ? p[base + i] : 0.0;
        a += loc[i];
    }
    part[threadIdx.x + 1] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        part[0] = boff[blockIdx.x];
        for (int t = 1; t <= 256; ++t) part[t] += part[t - 1];
    }
    __syncthreads();
    double run = part[threadIdx.x];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        run += loc[i];
        if (base + i < n) cdf[base + i] = run;
    }
}

cudaError_t launch_scan(const double *p, unsigned long long n, double *cdf, double *bsum, cudaStream_t st) {
    const long long nb = (long long)((n + SCAN_CHUNK - 1) / SCAN_CHUNK);
    scan_chunk_sums<<<(unsigned)nb, 256, 0, st>>>(p, n, bsum);
    scan_block_offsets<<<1, 256, 0, st>>>(bsum, nb);
    scan_chunk_apply<<<(unsigned)nb, 256, 0, st>>>(p, n, bsum, cdf);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- draws
__device__ __forceinline__ unsigned long long cdf_search(const double *cdf, unsigned long long n, double t) {
    // smallest i with cdf[i] > t; if none, the last i with a positive step
    if (!(cdf[n - 1] > t)) {
        unsigned long long i = n - 1;
        while (i > 0 && !(cdf[i] > cdf[i - 1])) --i;
        return i;
    }
    unsigned long long lo = 0, hi = n - 1;
    while (lo < hi) {
        const unsigned long long mid = lo + ((hi - lo) >> 1);
        if (cdf[mid] > t) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__global__ void draw_x_kernel(const double *cdf, int N, long long n_x, int mode, unsigned long long seed,
                              unsigned long long ctr0, unsigned long long *xs) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_x) return;
    const unsigned long long d = 1ULL << N;
    const double u = mc_uniform(seed, ctr0, (unsigned long long)i, 0ULL);
    unsigned long long x;
    if (i == 0) {
        x = 0ULL;          // x = 0 is its own stratum in both modes (SM Sec. I)
    } else if (mode == 0) {   // uniform on 1..d-1
        x = 1ULL + (unsigned long long)(u * (double)(d - 1));
        if (x >= d) x = d - 1;
    } else {                  // x ~ p(x | x != 0): inverse CDF over x >= 1
        const double c0 = cdf[0];
        x = cdf_search(cdf, d, c0 + u * (cdf[d - 1] - c0));
        if (x == 0) x = 1;
    }
    xs[i] = x;
}

cudaError_t launch_draw_x(const double *cdf, int N, long long n_x, int mode, unsigned long long seed,
                          unsigned long long ctr0, unsigned long long *xs, cudaStream_t st) {
    draw_x_kernel<<<(unsigned)((n_x + 255) / 256), 256, 0, st>>>(cdf, N, n_x, mode, seed, ctr0, xs);
    return cudaGetLastError();
}

// z-range selection: the FP32 range weights Wf[f][.] -> their inclusive FP64
// scan W[f][.] (fixed order), then each draw k picks range r and the
// remainder t' within it.
// First level of the z draw for one family per CTA. Thread t owns the
// contiguous ranges [t per, (t + 1) per) ("chunk" t). The FP64 CDF is
// C(i) = S_t + (w_lo + ... + w_i) for i in chunk t, summed in range order from
// the chunk's start S_t, where S_t is the inclusive scan of the chunk sums
// (each chunk summed as four interleaved partial sums, the scan by warp
// shuffles: short FP64 dependency chains on a narrow FP64 pipe). Draw k picks
// the chunk a with S_a <= t < S_{a+1}, t = u_k S_256, then the smallest range
// r of it with C(r) > t; if rounding leaves C below t at the chunk's end (or t
// reaches the total), the last range of positive weight is taken and its
// remainder is clamped by the sampler. It records t - C(r - 1) and the
// range's weight C(r) - C(r - 1). Rows of at most ZSEL_STAGE_MAX ranges (a
// power of two) are first staged in shared memory by coalesced loads, with
// one padding word per chunk so the chunk-wise reads are free of bank
// conflicts.
constexpr long long ZSEL_STAGE_MAX = 16384;
template <bool STAGED>
__global__ void __launch_bounds__(256) zrange_select_kernel(const float *Wf, long long nr, long long n_fam,
                                                            long long fam_base, int z_per_x, unsigned long long seed,
                                                            unsigned long long ctr0, DrawInfo *draws,
                                                            const unsigned long long *perm) {
    __shared__ double seg[257];     // seg[t] = S_t, seg[256] = the total
    __shared__ double wsum[8];
    extern __shared__ float swf[];
    const long long f = blockIdx.x;
    if (f >= n_fam) return;
    // the family's own index: its draw stream and its draw records
    const unsigned long long fam = perm ? perm[fam_base + f] : (unsigned long long)(fam_base + f);
    const long long per = (nr + 255) / 256;
    const float *wrow = Wf + (size_t)f * nr;
    const int lp = STAGED ? 31 - __clz((int)per) : 0;
    if constexpr (STAGED) {
        for (uint32_t i = threadIdx.x; i < (uint32_t)nr; i += 256) swf[i + (i >> lp)] = wrow[i];
        __syncthreads();
    }
    auto wf = [&](long long i) -> double {
        if constexpr (STAGED) return (double)swf[(uint32_t)i + ((uint32_t)i >> lp)];
        else return (double)wrow[i];
    };
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long lo = tid * per, hi = lo + per < nr ? lo + per : nr;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    long long i = lo;
    for (; i + 3 < hi; i += 4) {
        a0 += wf(i);
        a1 += wf(i + 1);
        a2 += wf(i + 2);
        a3 += wf(i + 3);
    }
    for (; i < hi; ++i) a0 += wf(i);
    double v = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double w = lane < 8 ? wsum[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const double u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        if (lane < 8) wsum[lane] = w;
    }
    __syncthreads();
    seg[tid + 1] = v + (warp > 0 ? wsum[warp - 1] : 0.0);
    if (tid == 0) seg[0] = 0.0;
    __syncthreads();
    const int tlast = (int)((nr - 1) / per);     // the last chunk that holds ranges
    const double total = seg[256];
    for (int k = tid; k < z_per_x; k += 256) {
        const double u = mc_uniform(seed, ctr0, fam, 1ULL + (unsigned long long)k);
        const double t = u * total;
        long long r = -1;
        double clo = 0.0, chi = 0.0;
        if (total > t) {
            int a = 0, b = tlast;                  // smallest a with S_{a+1} > t
            while (a < b) {
                const int mid = (a + b) >> 1;
                if (seg[mid + 1] > t) b = mid; else a = mid + 1;
            }
            const long long c0 = (long long)a * per, c1 = c0 + per < nr ? c0 + per : nr;
            double run = seg[a], lastp_lo = 0.0, lastp_hi = 0.0;
            long long lastp = -1;
            for (long long q = c0; q < c1; ++q) {
                const double w = wf(q), nrun = run + w;
                if (w > 0.0) { lastp = q; lastp_lo = run; lastp_hi = nrun; }
                if (nrun > t) { r = q; clo = run; chi = nrun; break; }
                run = nrun;
            }
            if (r < 0 && lastp >= 0) { r = lastp; clo = lastp_lo; chi = lastp_hi; }
        }
        if (r < 0) {
            // t at or past the total (or a chunk without weight): the last
            // range of positive weight
            for (int c = tlast; c >= 0 && r < 0; --c) {
                if (!(seg[c + 1] > seg[c])) continue;
                const long long c0 = (long long)c * per, c1 = c0 + per < nr ? c0 + per : nr;
                double run = seg[c];
                for (long long q = c0; q < c1; ++q) {
                    const double w = wf(q), nrun = run + w;
                    if (w > 0.0) { r = q; clo = run; chi = nrun; }
                    run = nrun;
                }
            }
            if (r < 0) { r = 0; clo = 0.0; chi = wf(0); }
        }
        DrawInfo di;
        di.range = (unsigned long long)r;
        di.t = t - clo;
        di.wr = chi - clo;
        di.pad = 0.0;
        draws[(size_t)fam * z_per_x + k] = di;
    }
}

cudaError_t launch_zrange_select(const float *Wf, long long nr, long long n_fam, long long fam_base, int z_per_x,
                                 unsigned long long seed, unsigned long long ctr0, DrawInfo *draws,
                                 const unsigned long long *perm, cudaStream_t st) {
    if (nr <= ZSEL_STAGE_MAX && (nr & (nr - 1)) == 0) {
        const size_t smem = sizeof(float) * (size_t)(nr + 256 + 1);
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(zrange_select_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(sizeof(float) * (ZSEL_STAGE_MAX + 257)));
            if (e != cudaSuccess) return e;
            attr = true;
        }
        zrange_select_kernel<true><<<(unsigned)n_fam, 256, smem, st>>>(Wf, nr, n_fam, fam_base, z_per_x, seed, ctr0,
                                                                       draws, perm);
    } else {
        zrange_select_kernel<false><<<(unsigned)n_fam, 256, 0, st>>>(Wf, nr, n_fam, fam_base, z_per_x, seed, ctr0,
                                                                     draws, perm);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ MC statistics
// Per family i: y[i][0..2] = mean over its z-draws of (-log2 c^2, c^2, c^4);
// y[i][3..5] = the family's exact conditional means (-sum c^2 log2 c^2,
// sum c^4, sum c^6) / sum c^2 (marginal mode; family 0, the x = 0 stratum,
// takes the exact means in both slots), or, uniform mode, the SM Sec. I
// family values h_x, m_{2;x}, m_{3;x} in y[i][0..2].
__global__ void mc_family_stats_kernel(const FamMoments *fm, const float *cz, long long n_x, int z_per_x, int N,
                                       int mode, double *y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_x) return;
    const double d = ldexp(1.0, N);
    const FamMoments &m = fm[i];
    double *o = y + 6 * i;
    if (mode == 0) {
        o[0] = N * (m.m[0] / d) - m.m[3] / d;
        o[1] = m.m[1] / (d * d);
        o[2] = m.m[2] / (d * d * d);
        o[3] = o[4] = o[5] = 0.0;
    } else {
        double a0 = 0, a1 = 0, a2 = 0;
        for (int k = 0; k < z_per_x; ++k) {
            const double c = (double)cz[(size_t)i * z_per_x + k];
            const double c2 = c * c;
            a0 += -log2(c2);
            a1 += c2;
            a2 += c2 * c2;
        }
        o[3] = -m.m[3] / m.m[0]; o[4] = m.m[1] / m.m[0]; o[5] = m.m[2] / m.m[0];
        if (i == 0) { o[0] = o[3]; o[1] = o[4]; o[2] = o[5]; }
        else { o[0] = a0 / z_per_x; o[1] = a1 / z_per_x; o[2] = a2 / z_per_x; }
    }
}

// out[0..5] = sum_{i >= first} y[i][a], out[6..11] = sum y^2, out[12..17] = y[0][a],
// out[18] = sum over families of sum c^2 / (d p(x)) estimate (marginal) -- fixed order.
__global__ void __launch_bounds__(256) mc_totals_kernel(const double *y, long long n_x, int first,
                                                        const FamMoments *fm, double *out) {
    __shared__ double red[8];
    for (int a = 0; a < 6; ++a) {
        NeuSum ns, nq;
        for (long long i = first + threadIdx.x; i < n_x; i += 256) {
            const double v = y[6 * i + a];
            ns.add(v);
            nq.add(v * v);
        }
        const double s = block_sum<256>(ns.value(), red);
        const double q = block_sum<256>(nq.value(), red);
        if (threadIdx.x == 0) { out[a] = s; out[6 + a] = q; out[12 + a] = y[a]; }
    }
    NeuSum np_;
    for (long long i = threadIdx.x; i < n_x; i += 256) np_.add(fm[i].m[0]);
    const double p = block_sum<256>(np_.value(), red);
    if (threadIdx.x == 0) out[18] = p;
}

cudaError_t launch_mc_stats(const FamMoments *fm, const float *cz, long long n_x, int z_per_x, int N, int mode,
                            double *y, double *out, cudaStream_t st) {
    mc_family_stats_kernel<<<(unsigned)((n_x + 127) / 128), 128, 0, st>>>(fm, cz, n_x, z_per_x, N, mode, y);
    mc_totals_kernel<<<1, 256, 0, st>>>(y, n_x, 1, fm, out);
    return cudaGetLastError();
}

// ------------------------------------------------------- batched states
// per-state sum |psi|^2: grid (blocks per state, states), fixed order
__global__ void __launch_bounds__(256) norm2_multi_partial(const float2 *const *psi_list, int N, int nb,
                                                           double *partial) {
    __shared__ double red[8];
    const int st = blockIdx.y;
    const float2 *psi = psi_list[st];
    const unsigned long long d = 1ULL << N;
    double acc = 0.0;
    const unsigned long long stride = (unsigned long long)nb * blockDim.x;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; b < d; b += stride) {
        const float2 u = __ldg(psi + b);
        const double ux = f2d(u.x), uy = f2d(u.y);
        acc = fma(ux, ux, acc);
        acc = fma(uy, uy, acc);
    }
    acc = block_sum<256>(acc, red);
    if (threadIdx.x == 0) partial[(size_t)st * nb + blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) norm2_multi_final(const double *partial, int nb, double *norm2, double *s) {
    __shared__ double red[8];
    const int st = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) acc += partial[(size_t)st * nb + i];
    acc = block_sum<256>(acc, red);
    if (threadIdx.x == 0) {
        norm2[st] = acc;
        s[st] = acc > 0.0 ? 1.0 / acc : 0.0;
    }
}

cudaError_t launch_norm2_multi(const float2 *const *psi_list, int n_states, int N, double *partial, int nb,
                               double *norm2, double *s, cudaStream_t st) {
    norm2_multi_partial<<<dim3(nb, n_states), 256, 0, st>>>(psi_list, N, nb, partial);
    norm2_multi_final<<<n_states, 256, 0, st>>>(partial, nb, norm2, s);
    return cudaGetLastError();
}

// per-state totals of the family sums of states [s0, s0 + ns): one block per
// state over its 2^N consecutive families (fixed order); candidate families
// appended to flags as F = (state << N) | x.
__global__ void __launch_bounds__(256) state_totals_kernel(const FamMoments *fm, long long fm_first_family, int N,
                                                           int s0, double *totals, unsigned long long *flags,
                                                           unsigned long long *n_flag) {
    __shared__ double red[8];
    const int st = s0 + blockIdx.x;
    const long long nf = 1LL << N;
    const long long f0 = ((long long)st << N) - fm_first_family;
    NeuSum n0, n1, n2, n3, nq;
    double c = 0;
    for (long long f = threadIdx.x; f < nf; f += 256) {
        const FamMoments &m = fm[f0 + f];
        n0.add(m.m[0]); n1.add(m.m[1]); n2.add(m.m[2]); n3.add(m.m[3]); c += (double)m.cand;
        if (f > 0) nq.add(m.m[1] * m.m[1]);
        if (m.cand) {
            const unsigned long long pos = atomicAdd(n_flag, 1ULL);
            flags[pos] = ((unsigned long long)st << N) | (unsigned long long)f;
        }
    }
    double a0 = n0.value(), a1 = n1.value(), a2 = n2.value(), a3 = n3.value(), q = nq.value();
    a0 = block_sum<256>(a0, red);
    a1 = block_sum<256>(a1, red);
    a2 = block_sum<256>(a2, red);
    a3 = block_sum<256>(a3, red);
    c = block_sum<256>(c, red);
    q = block_sum<256>(q, red);
    if (threadIdx.x == 0) {
        double *o = totals + TOT_N * (size_t)st;
        o[0] = a0; o[1] = a1; o[2] = a2; o[3] = a3; o[4] = c; o[5] = q; o[6] = fm[f0].m[1];
    }
}

cudaError_t launch_state_totals(const FamMoments *fm, long long fm_first_family, int N, int s0, int ns,
                                double *totals, unsigned long long *flags, unsigned long long *n_flag,
                                cudaStream_t st) {
    state_totals_kernel<<<ns, 256, 0, st>>>(fm, fm_first_family, N, s0, totals, flags, n_flag);
    return cudaGetLastError();
}

// stab counts of flagged families added to their states (integer atomics)
__global__ void count_scatter_kernel(const unsigned long long *flags, const unsigned long long *counts, long long n,
                                     int N, unsigned long long *state_count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (counts[i]) atomicAdd(state_count + (flags[i] >> N), counts[i]);
}

cudaError_t launch_count_scatter(const unsigned long long *flags, const unsigned long long *counts, long long n,
                                 int N, unsigned long long *state_count, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    count_scatter_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(flags, counts, n, N, state_count);
    return cudaGetLastError();
}

cudaError_t launch_philox_test(const unsigned long long *ctr_key, unsigned long long *out, int n, cudaStream_t st) {
    philox_test_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctr_key, out, n);
    return cudaGetLastError();
}

} // namespace sre
