// k_null.cu -- FP64 recount of nullity-candidate families at their listed z.
//
// The stabilizer count of Algorithm 1 is #{P : | |c_P| - 1 | < eps}, decided
// in FP64. A family flagged by the FP32 sweep (some |c| near 1) is recounted
// at the packed z' an FP32 candidate pass listed for it: every other z' holds
// only |c| below the candidate threshold, which lies more than 1e-4 (far
// beyond the FP32 error) under 1 - eps. For the listed z',
//   H(z') = sum_g h(g) (-1)^{popc(g & z')},   g < 2^(N-1),
// with h(g) = conj psi(b ^ x) psi(b), b = g with 0 inserted at bit j (the top
// bit of x), or h(g) = (|psi(g)|^2, |psi(g + 2^(N-1))|^2) for x = 0: the same
// packed transform the sweep evaluates, here one output at a time. The pair
// (c(z0), c(z1)) follows from H(z') as in the transform (up to signs, which
// the count ignores). Each family costs 2^(N-1) (4 + 2k) FP64 operations for k
// listed z', against about 2^(N-1) (2N + 8) for a full FP64 transform, so
// families with more than kdirect candidates are appended to an overflow list
// and recounted by the transform instead.
#include "k_misc.cuh"

namespace sre {

namespace {

constexpr int ND_THREADS = 256;
constexpr int ND_GROUP = 8;      // z' summed per sweep over g

// v with its sign bit flipped when sgn = 1u << 31
__device__ __forceinline__ double flip(double v, unsigned sgn) {
    return __hiloint2double(__double2hiint(v) ^ (int)sgn, __double2loint(v));
}

template <int G>
__device__ __forceinline__ void direct_sums(const float2 *psi, uint32_t x, int j, uint32_t half,
                                            const uint32_t (&zl)[ND_GROUP], double (&ar)[ND_GROUP],
                                            double (&ai)[ND_GROUP]) {
#pragma unroll 2
    for (uint32_t g = threadIdx.x; g < half; g += ND_THREADS) {
        double hr, hi;
        if (x) {
            const uint32_t b = (uint32_t)insert0(g, j);
            const float2 u = __ldg(psi + b), w = __ldg(psi + (b ^ x));
            const double ux = u.x, uy = u.y, wx = w.x, wy = w.y;
            hr = fma(wx, ux, wy * uy);
            hi = fma(wx, uy, -(wy * ux));
        } else {
            const float2 u = __ldg(psi + g), w = __ldg(psi + (g + half));
            const double ux = u.x, uy = u.y, wx = w.x, wy = w.y;
            hr = fma(ux, ux, uy * uy);
            hi = fma(wx, wx, wy * wy);
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const unsigned sgn = (unsigned)(__popc(g & zl[i]) & 1) << 31;
            ar[i] += flip(hr, sgn);
            ai[i] += flip(hi, sgn);
        }
    }
}

__global__ void __launch_bounds__(ND_THREADS) null_direct_kernel(const NullDirectArgs a) {
    __shared__ uint32_t zs[NULL_CAND_MAX];
    __shared__ double red[ND_THREADS / 32][2 * ND_GROUP];
    const long long slot = blockIdx.x;
    const unsigned cnt = a.cand_cnt[slot];
    const unsigned long long F = a.xs[a.fam_base + slot];
    if (cnt == 0 || cnt > (unsigned)a.kdirect) {
        if (threadIdx.x == 0) {
            a.counts[slot] = 0;
            if (cnt) a.ovf[atomicAdd(a.ovf_n, 1ULL)] = F;
        }
        return;
    }
    const int N = a.N;
    const uint32_t x = (uint32_t)(F & ((1ULL << N) - 1ULL));
    const float2 *psi = a.psi;
    const double *s_ptr = a.s_ptr;
    if (a.psi_list) {
        psi = a.psi_list[F >> N];
        s_ptr = a.s_list + (F >> N);
    }
    const uint32_t half = 1u << (N - 1);
    const int j = x ? 31 - __clz((int)x) : N - 1;
    for (unsigned i = threadIdx.x; i < cnt; i += ND_THREADS) zs[i] = a.cand_z[(size_t)slot * a.cand_max + i];
    __syncthreads();
    const double s = *s_ptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long total = 0;
    for (unsigned g0 = 0; g0 < cnt; g0 += ND_GROUP) {
        const int ng = (int)min((unsigned)ND_GROUP, cnt - g0);
        uint32_t zl[ND_GROUP];
        double ar[ND_GROUP], ai[ND_GROUP];
#pragma unroll
        for (int i = 0; i < ND_GROUP; ++i) {
            zl[i] = i < ng ? zs[g0 + i] : 0u;
            ar[i] = 0.0;
            ai[i] = 0.0;
        }
        switch (ng) {
        case 1: direct_sums<1>(psi, x, j, half, zl, ar, ai); break;
        case 2: direct_sums<2>(psi, x, j, half, zl, ar, ai); break;
        case 3: direct_sums<3>(psi, x, j, half, zl, ar, ai); break;
        case 4: direct_sums<4>(psi, x, j, half, zl, ar, ai); break;
        case 5: direct_sums<5>(psi, x, j, half, zl, ar, ai); break;
        case 6: direct_sums<6>(psi, x, j, half, zl, ar, ai); break;
        case 7: direct_sums<7>(psi, x, j, half, zl, ar, ai); break;
        default: direct_sums<8>(psi, x, j, half, zl, ar, ai); break;
        }
        // fixed-order block sums: warp butterflies, then the warps in order
#pragma unroll
        for (int i = 0; i < ND_GROUP; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ar[i] += __shfl_xor_sync(0xffffffffu, ar[i], o);
                ai[i] += __shfl_xor_sync(0xffffffffu, ai[i], o);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < ND_GROUP; ++i) {
                red[warp][i] = ar[i];
                red[warp][ND_GROUP + i] = ai[i];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 0; i < ng; ++i) {
                double hr = 0.0, hi = 0.0;
                for (int w = 0; w < ND_THREADS / 32; ++w) {
                    hr += red[w][i];
                    hi += red[w][ND_GROUP + i];
                }
                double c0, c1;
                if (x) { c0 = 2.0 * s * hr; c1 = 2.0 * s * hi; }
                else { c0 = s * (hr + hi); c1 = s * (hr - hi); }
                total += (fabs(fabs(c0) - 1.0) < a.eps) ? 1ULL : 0ULL;
                total += (fabs(fabs(c1) - 1.0) < a.eps) ? 1ULL : 0ULL;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) a.counts[slot] = total;
}

} // namespace

cudaError_t launch_null_direct(const NullDirectArgs &a, long long n_fam, cudaStream_t st) {
    if (n_fam <= 0) return cudaSuccess;
    if (n_fam > 0x7fffffffLL || a.N < 1 || a.N > 31 || a.kdirect > NULL_CAND_MAX || a.kdirect > a.cand_max)
        return cudaErrorInvalidValue;
    null_direct_kernel<<<(unsigned)n_fam, ND_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

} // namespace sre
