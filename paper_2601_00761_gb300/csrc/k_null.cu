// k_null.cu -- FP64 recount of nullity-candidate families at their listed z.
//
// The stabilizer count of Algorithm 1 is #{P : | |c_P| - 1 | < eps}, decided
// in FP64. A family flagged by the FP32 sweep (some |c| near 1) is recounted
// at the packed z' an FP32 candidate pass listed for it: every other z' holds
// only |c| below the candidate threshold, which lies more than 1e-4 (far
// beyond the FP32 error) under 1 - eps. For a packed z',
//   H(z') = sum_g h(g) (-1)^{popc(g & z')},   g < 2^(N-1),
// with h(g) = conj psi(b ^ x) psi(b), b = g with 0 inserted at bit j (the top
// bit of x), or h(g) = (|psi(g)|^2, |psi(g + 2^(N-1))|^2) for x = 0: the same
// packed transform the sweep evaluates, here at chosen outputs. The pair
// (c(z0), c(z1)) follows from H(z') as in the transform (up to signs, which
// the count ignores). Routes, per family (one CTA each):
//  - coset: the listed z' lie in z'_0 + span(v_1..v_m), m <= 6 (stabilizer
//    structure). One sweep over g accumulates h(g) (-1)^{g.z'_0} into 2^m bins
//    keyed by the parities g.v_i, and an m-bit WHT of the bins gives H on the
//    whole coset: 6 FP64 operations per point for any number of candidates.
//  - direct: wider spans with at most kdirect candidates: H at each listed z'
//    by its own signed sum, 4 + 2k operations per point for k candidates.
//  - overflow: the rest (or more than cand_max candidates, the list then being
//    incomplete) is appended to a list for the FP64 transform, about 2N + 12
//    operations per point.
// Points of a coset that were not listed lie below the threshold and count
// nothing, so every route counts exactly the FP64 decisions.
#include "k_misc.cuh"
#include "k_fp64.cuh"

namespace sre {

namespace {

constexpr int ND_THREADS = 256;
constexpr int ND_GROUP = 8;      // z' summed per sweep over g (direct route)
constexpr int NB_CHUNK = 16;     // bins accumulated per sweep over g (coset route)
constexpr int NB_MAXBITS = 6;    // span dimension up to which the coset route is taken

// v with its sign bit flipped when sgn = 1u << 31
__device__ __forceinline__ double flip(double v, unsigned sgn) {
    return __hiloint2double(__double2hiint(v) ^ (int)sgn, __double2loint(v));
}

// h(g) in FP64 (exact products of the FP32 amplitudes, one rounding per sum)
__device__ __forceinline__ void hval(const float2 *psi, uint32_t x, int j, uint32_t half, uint32_t g, double &hr,
                                     double &hi) {
    if (x) {
        const uint32_t b = (uint32_t)insert0(g, j);
        const float2 u = __ldg(psi + b), w = __ldg(psi + (b ^ x));
        const double ux = f2d(u.x), uy = f2d(u.y), wx = f2d(w.x), wy = f2d(w.y);
        hr = fma(wx, ux, wy * uy);
        hi = fma(wx, uy, -(wy * ux));
    } else {
        const float2 u = __ldg(psi + g), w = __ldg(psi + (g + half));
        const double ux = f2d(u.x), uy = f2d(u.y), wx = f2d(w.x), wy = f2d(w.y);
        hr = fma(ux, ux, uy * uy);
        hi = fma(wx, wx, wy * wy);
    }
}

// direct route: H at G listed z' per sweep over all g
template <int G>
__device__ __forceinline__ void direct_sums(const float2 *psi, uint32_t x, int j, uint32_t half,
                                            const uint32_t (&zl)[ND_GROUP], double (&ar)[ND_GROUP],
                                            double (&ai)[ND_GROUP]) {
#pragma unroll 2
    for (uint32_t g = threadIdx.x; g < half; g += ND_THREADS) {
        double hr, hi;
        hval(psi, x, j, half, g, hr, hi);
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const unsigned sgn = (unsigned)(__popc(g & zl[i]) & 1) << 31;
            ar[i] += flip(hr, sgn);
            ai[i] += flip(hi, sgn);
        }
    }
}

// coset route: the candidates lie in z0 + span(v_0 .. v_{m-1}), the v_i
// reduced (v_i holds pivot bit piv_i and no other pivot), pivots ascending.
// Bin b collects h(g) (-1)^{popc(g & z0)} over the g with parity(g & v_i) =
// b_i; then H(z0 + sum_i a_i v_i) = sum_b bin_b (-1)^{a.b}. With g = r (bits
// spread over the non-pivot positions) | t (pivot bits), parity(g & v_i) =
// c_i(r) ^ t_i, so each r meets every bin exactly once. This sweep covers the
// 2^MB bins whose high bits (basis vectors MB .. m-1) are fixed by offq.
template <int MB>
__device__ __forceinline__ void coset_sums(const float2 *psi, uint32_t x, int j, uint32_t half, uint32_t z0,
                                           const uint32_t *vb, const uint32_t *piv, int m, uint32_t offq,
                                           double (&ar)[NB_CHUNK], double (&ai)[NB_CHUNK]) {
    constexpr int NBIN = 1 << MB;
    uint32_t offl[NBIN];
#pragma unroll
    for (int b = 0; b < NBIN; ++b) {
        uint32_t o = 0;
#pragma unroll
        for (int i = 0; i < MB; ++i)
            if ((b >> i) & 1) o |= 1u << piv[i];
        offl[b] = o;
    }
    const uint32_t nr = half >> m;
    for (uint32_t r = threadIdx.x; r < nr; r += ND_THREADS) {
        uint32_t gr = r, C = 0;
        for (int i = 0; i < m; ++i) gr = (uint32_t)insert0(gr, (int)piv[i]);
        for (int i = 0; i < m; ++i) C |= (uint32_t)(__popc(gr & vb[i]) & 1) << piv[i];
        const uint32_t G0 = gr ^ C ^ offq;
#pragma unroll
        for (int b = 0; b < NBIN; ++b) {
            const uint32_t g = G0 ^ offl[b];
            double hr, hi;
            hval(psi, x, j, half, g, hr, hi);
            const unsigned sgn = (unsigned)(__popc(g & z0) & 1) << 31;
            ar[b] += flip(hr, sgn);
            ai[b] += flip(hi, sgn);
        }
    }
}

// fixed-order block sums of the first n (<= NB_CHUNK) pairs (ar, ai): warp
// butterflies, then the warps in order; the sums land in out_r/out_i[0..n)
template <int NV>
__device__ __forceinline__ void block_sums(double (&ar)[NV], double (&ai)[NV], int n, double (*red)[2 * NB_CHUNK],
                                           double *out_r, double *out_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ar[i] += __shfl_xor_sync(0xffffffffu, ar[i], o);
            ai[i] += __shfl_xor_sync(0xffffffffu, ai[i], o);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            red[warp][i] = ar[i];
            red[warp][NB_CHUNK + i] = ai[i];
        }
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t < 2 * n) {
        const int i = t < n ? t : t - n, col = t < n ? i : NB_CHUNK + i;
        double v = 0.0;
        for (int w = 0; w < ND_THREADS / 32; ++w) v += red[w][col];
        if (t < n) out_r[i] = v;
        else out_i[i] = v;
    }
    __syncthreads();
}

// the two expectations of the pair H(z') yields, decided in FP64
__device__ __forceinline__ int count_pair(double hr, double hi, bool xnz, double s, double eps) {
    double c0, c1;
    if (xnz) { c0 = 2.0 * s * hr; c1 = 2.0 * s * hi; }
    else { c0 = s * (hr + hi); c1 = s * (hr - hi); }
    return (fabs(fabs(c0) - 1.0) < eps ? 1 : 0) + (fabs(fabs(c1) - 1.0) < eps ? 1 : 0);
}

enum { NR_COSET = 0, NR_DIRECT = 1, NR_OVERFLOW = 2 };

__global__ void __launch_bounds__(ND_THREADS) null_direct_kernel(const NullDirectArgs a) {
    __shared__ uint32_t zs[NULL_CAND_MAX];
    __shared__ uint32_t vb[NB_MAXBITS], piv[NB_MAXBITS];
    __shared__ int s_mode, s_m;
    __shared__ double red[ND_THREADS / 32][2 * NB_CHUNK];
    __shared__ double bin_r[1 << NB_MAXBITS], bin_i[1 << NB_MAXBITS];
    const long long slot = blockIdx.x;
    const unsigned cnt = a.cand_cnt[slot];
    const unsigned long long F = a.xs[a.fam_base + slot];
    if (cnt == 0 || cnt > (unsigned)a.cand_max) {     // nothing to count, or the list is incomplete
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
    if (threadIdx.x == 0) {
        // reduced basis of span{z_i ^ z_0} (GF(2) elimination, highest bit as pivot)
        uint32_t bv[NB_MAXBITS + 1], bp[NB_MAXBITS + 1];
        int m = 0;
        bool wide = false;
        for (unsigned i = 1; i < cnt && !wide; ++i) {
            uint32_t u = zs[i] ^ zs[0];
            for (int l = 0; l < m; ++l)
                if ((u >> bp[l]) & 1u) u ^= bv[l];
            if (!u) continue;
            if (m == NB_MAXBITS) { wide = true; break; }
            const uint32_t p = 31u - (uint32_t)__clz((int)u);
            for (int l = 0; l < m; ++l)
                if ((bv[l] >> p) & 1u) bv[l] ^= u;
            bv[m] = u;
            bp[m] = p;
            ++m;
        }
        if (!wide) {
            for (int l = 1; l < m; ++l)          // pivots ascending
                for (int q = l; q > 0 && bp[q - 1] > bp[q]; --q) {
                    const uint32_t tv = bv[q], tp = bp[q];
                    bv[q] = bv[q - 1]; bp[q] = bp[q - 1];
                    bv[q - 1] = tv; bp[q - 1] = tp;
                }
            for (int l = 0; l < m; ++l) { vb[l] = bv[l]; piv[l] = bp[l]; }
            s_mode = NR_COSET;
            s_m = m;
        } else {
            s_mode = cnt <= (unsigned)a.kdirect ? NR_DIRECT : NR_OVERFLOW;
            s_m = 0;
        }
    }
    __syncthreads();
    const int mode = s_mode, m = s_m;
    if (mode == NR_OVERFLOW) {
        if (threadIdx.x == 0) {
            a.counts[slot] = 0;
            a.ovf[atomicAdd(a.ovf_n, 1ULL)] = F;
        }
        return;
    }
    const double s = *s_ptr;
    int total = 0;
    if (mode == NR_COSET) {
        const uint32_t z0 = zs[0];
        const int MBv = m < 4 ? m : 4;
        const int nq = 1 << (m - MBv);
        for (int q = 0; q < nq; ++q) {
            uint32_t offq = 0;
            for (int i = 0; i < m - MBv; ++i)
                if ((q >> i) & 1) offq |= 1u << piv[MBv + i];
            double ar[NB_CHUNK], ai[NB_CHUNK];
#pragma unroll
            for (int b = 0; b < NB_CHUNK; ++b) { ar[b] = 0.0; ai[b] = 0.0; }
            switch (MBv) {
            case 0: coset_sums<0>(psi, x, j, half, z0, vb, piv, m, offq, ar, ai); break;
            case 1: coset_sums<1>(psi, x, j, half, z0, vb, piv, m, offq, ar, ai); break;
            case 2: coset_sums<2>(psi, x, j, half, z0, vb, piv, m, offq, ar, ai); break;
            case 3: coset_sums<3>(psi, x, j, half, z0, vb, piv, m, offq, ar, ai); break;
            default: coset_sums<4>(psi, x, j, half, z0, vb, piv, m, offq, ar, ai); break;
            }
            block_sums<NB_CHUNK>(ar, ai, 1 << MBv, red, bin_r + (q << MBv), bin_i + (q << MBv));
        }
        // m-bit transform of the bins: H(z0 + sum_i a_i v_i) for every a
        const int t = threadIdx.x, nb = 1 << m;
        for (int st = 0; st < m; ++st) {
            double vr = 0.0, vi = 0.0;
            if (t < nb) {
                const int p = t ^ (1 << st);
                if (t & (1 << st)) { vr = bin_r[p] - bin_r[t]; vi = bin_i[p] - bin_i[t]; }
                else { vr = bin_r[t] + bin_r[p]; vi = bin_i[t] + bin_i[p]; }
            }
            __syncthreads();
            if (t < nb) { bin_r[t] = vr; bin_i[t] = vi; }
            __syncthreads();
        }
        const int c = t < nb ? count_pair(bin_r[t], bin_i[t], x != 0, s, a.eps) : 0;
        total = __syncthreads_count(c >= 1) + __syncthreads_count(c == 2);
    } else {
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
            block_sums<ND_GROUP>(ar, ai, ng, red, bin_r, bin_i);
            const int t = threadIdx.x;
            const int c = t < ng ? count_pair(bin_r[t], bin_i[t], x != 0, s, a.eps) : 0;
            total += __syncthreads_count(c >= 1) + __syncthreads_count(c == 2);
        }
    }
    if (threadIdx.x == 0) a.counts[slot] = (unsigned long long)total;
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
