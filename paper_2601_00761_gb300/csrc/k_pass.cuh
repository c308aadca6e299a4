// k_pass.cuh -- the transform pass kernel template and its launcher.
//
// One kernel template serves every pass of every transform in the library:
//   prologue  SRC_PSI_FAMILY : h(b') = conj(psi[b^x]) psi[b], b = b' with 0 at bit j
//             SRC_PSI_Q      : h(g)  = (|psi[g]|^2, |psi[g + d/2]|^2)  (x = 0 family / marginal)
//             SRC_BUF        : the previous pass's output
//             SRC_GRAM       : h(a) = C[a][a ^ x] of a reduced state (C = Psi Psi^H)
//   epilogue  DST_BUF        : store for the next pass
//             DST_MOMENTS    : fused reduction of Algorithm 1 (sum c^2, c^4, c^6,
//                              c^2 log2 c^2, FP32 nullity candidates, z-range weights)
//             DST_SPECTRUM   : c_{x,z} for every z
//             DST_NULLCOUNT  : #{z : | |c| - 1 | < eps} (FP64 recheck)
//             DST_SQMAP/DST_P: the two elementwise maps of the x-marginal
// The tile geometry (M, LO) and the element type are template parameters; the
// pass's global bit offset and the family come from PassArgs / the grid.
#pragma once

#include "sre_internal.cuh"
#include "k_tc.cuh"

namespace sre {

__device__ __forceinline__ int sgn_phase(int k) { return (((k + 1) >> 1) & 1) ? -1 : 1; }

// Sum over the T threads of a group; the result is valid in the group's thread 0.
// red: shared scratch of at least NT/32 doubles. All threads of the CTA call it.
template <int T, int NT>
__device__ __forceinline__ double group_sum(double v, double *red) {
    if constexpr (T >= 32) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if constexpr (T == 32) {
            return v;
        } else {
            const int w = threadIdx.x >> 5;
            __syncthreads();
            if ((threadIdx.x & 31) == 0) red[w] = v;
            __syncthreads();
            double s = 0.0;
            if ((threadIdx.x & (T - 1)) == 0) {
#pragma unroll 1
                for (int i = 0; i < T / 32; ++i) s += red[w + i];
            }
            return s;
        }
    } else {
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
}

// NV sums and one maximum over the T threads of a group: FP32 butterfly
// inside the warp, FP64 butterfly across the group's warps. Results are valid
// in the group's thread 0. red: (NV + 1) * NT/32 floats of shared scratch.
// Two barriers when a group spans several warps.
//
// The cross-warp step runs in the group's first warp with one lane per
// (value, warp) pair, so the whole tile costs a handful of FP64 warp
// instructions: the FP64 pipe issues one warp instruction per 16 cycles on
// this part, and a serial per-value loop in one thread would sit on the
// critical path of every tile.
template <int T, int NT, int NV>
__device__ __forceinline__ void group_reduce(float (&v)[NV], float &mx, double (&out)[NV], float &omx,
                                             double *red) {
    constexpr int W = T < 32 ? T : 32;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if constexpr (T <= 32) {
#pragma unroll
        for (int i = 0; i < NV; ++i) out[i] = (double)v[i];
        omx = mx;
    } else {
        constexpr int NW = NT / 32;          // warps in the CTA
        constexpr int WPG = T / 32;          // warps per group (power of two, <= 32)
        constexpr int VPP = 32 / WPG;        // values reduced per round by one warp
        constexpr int NVM = NV + 1;          // the sums and the maximum
        constexpr int ROUNDS = (NVM + VPP - 1) / VPP;
        float *rf = reinterpret_cast<float *>(red);
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        __syncthreads();
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < NV; ++i) rf[i * NW + w] = v[i];
            rf[NV * NW + w] = mx;
        }
        __syncthreads();
        if ((w & (WPG - 1)) == 0) {
            const int q = lane & (WPG - 1), vi = lane / WPG;
#pragma unroll
            for (int r = 0; r < ROUNDS; ++r) {
                const int vv = r * VPP + vi;
                const float f = vv < NVM ? rf[vv * NW + w + q] : 0.f;
                double sd = (double)f;
                float sm = f;
#pragma unroll
                for (int o = WPG / 2; o > 0; o >>= 1) {
                    sd += __shfl_xor_sync(0xffffffffu, sd, o);
                    sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
                }
#pragma unroll
                for (int u = 0; u < VPP; ++u) {
                    const int idx = r * VPP + u;
                    if (idx < NV) out[idx] = __shfl_sync(0xffffffffu, sd, u * WPG);
                    else if (idx == NV) omx = __shfl_sync(0xffffffffu, sm, u * WPG);
                }
            }
        }
    }
}

// bit k of the result = parity(a & k), k < 32 (the Walsh function of a)
__device__ __forceinline__ uint32_t walsh_mask5(uint32_t a) {
    uint32_t m = 0;
    if (a & 1u) m ^= 0xAAAAAAAAu;
    if (a & 2u) m ^= 0xCCCCCCCCu;
    if (a & 4u) m ^= 0xF0F0F0F0u;
    if (a & 8u) m ^= 0xFF00FF00u;
    if (a & 16u) m ^= 0xFFFF0000u;
    return m;
}

// 32-bit packed global indices of a thread's slots (N <= 31, so every packed
// index and every psi index is below 2^31). The thread's slot-0 index is
// base; slot k of the mapping whose slot bits start at tile bit A adds the
// column part of k << A and its row part times 2^lo_g (all bit fields
// disjoint, so the OR of the fields is their sum).
template <class Cfg>
__device__ __forceinline__ uint32_t thread_gidx(unsigned long long gbase, int lo_g, uint32_t e) {
    return (uint32_t)gbase | ((e >> Cfg::LO) << lo_g) | (e & ((1u << Cfg::LO) - 1u));
}
template <class Cfg, int A>
__device__ __forceinline__ uint32_t slot_gidx(uint32_t base, uint32_t rs, int k) {
    constexpr uint32_t CM = (1u << Cfg::LO) - 1u;
    const uint32_t e = (uint32_t)k << A;
    return base + (e & CM) + (e >> Cfg::LO) * rs;
}

// Load the tile in the first round's mapping (prologue of every pass).
template <class Cfg, int SRC>
__device__ __forceinline__ void pass_prologue(typename Cfg::C2 (&v)[Cfg::E], const PassArgs &a, const float2 *psi,
                                              long long slot, unsigned long long x, int j, unsigned long long half,
                                              unsigned long long gbase, uint32_t t) {
    typedef typename Cfg::Real R;
    typedef typename Cfg::C2 C2;
    constexpr int A0 = Maps<Cfg>::first;
    const uint32_t base = thread_gidx<Cfg>(gbase, a.lo_g, Cfg::elem(t, 0, A0));
    const uint32_t rs = 1u << a.lo_g;
    if constexpr (SRC == SRC_PSI_FAMILY) {
        // loads issued in batches of LB slots (2 LB independent 8-byte loads in
        // flight per thread) before any of them is used
        constexpr int LB = Cfg::E < 8 ? Cfg::E : 8;
        if (x != 0) {
            // b = g with 0 inserted at bit j = g + (g & ~(2^j - 1)); partner b ^ x
            const uint32_t hm = ~((1u << j) - 1u), x32 = (uint32_t)x;
#pragma unroll
            for (int k0 = 0; k0 < Cfg::E; k0 += LB) {
                float2 u[LB], w[LB];
#pragma unroll
                for (int q = 0; q < LB; ++q) {
                    const uint32_t g = slot_gidx<Cfg, A0>(base, rs, k0 + q);
                    const uint32_t b = g + (g & hm);
                    u[q] = __ldg(psi + b);
                    w[q] = __ldg(psi + (b ^ x32));
                }
#pragma unroll
                for (int q = 0; q < LB; ++q) {
                    const R ux = u[q].x, uy = u[q].y, wx = w[q].x, wy = w[q].y;
                    v[k0 + q].x = fma(wx, ux, wy * uy);     // conj(w) * u, contraction fixed
                    v[k0 + q].y = fma(wx, uy, -(wy * ux));
                }
            }
        } else {
            const uint32_t h32 = (uint32_t)half;
#pragma unroll
            for (int k0 = 0; k0 < Cfg::E; k0 += LB) {
                float2 u[LB], w[LB];
#pragma unroll
                for (int q = 0; q < LB; ++q) {
                    const uint32_t g = slot_gidx<Cfg, A0>(base, rs, k0 + q);
                    u[q] = __ldg(psi + g);
                    w[q] = __ldg(psi + (g | h32));
                }
#pragma unroll
                for (int q = 0; q < LB; ++q) {
                    const R ux = u[q].x, uy = u[q].y, wx = w[q].x, wy = w[q].y;
                    v[k0 + q].x = fma(ux, ux, uy * uy);
                    v[k0 + q].y = fma(wx, wx, wy * wy);
                }
            }
        }
    } else if constexpr (SRC == SRC_GRAM) {
        // h(a) = sum_e conj(psi(a ^ x, e)) psi(a, e) = C[a][a ^ x]; x = 0: the
        // diagonal pair (C[g][g], C[g + d/2][g + d/2])
        const float2 *C = a.gram;
        const unsigned long long ld = (unsigned long long)a.gram_ld;
        if (x != 0) {
            const uint32_t hm = ~((1u << j) - 1u), x32 = (uint32_t)x;
#pragma unroll
            for (int k = 0; k < Cfg::E; ++k) {
                const uint32_t g = slot_gidx<Cfg, A0>(base, rs, k);
                const uint32_t r = g + (g & hm);
                const float2 h = __ldg(C + r + ld * (r ^ x32));
                v[k].x = h.x;
                v[k].y = h.y;
            }
        } else {
            const uint32_t h32 = (uint32_t)half;
#pragma unroll
            for (int k = 0; k < Cfg::E; ++k) {
                const uint32_t g = slot_gidx<Cfg, A0>(base, rs, k), gh = g | h32;
                v[k].x = __ldg(C + g + ld * g).x;
                v[k].y = __ldg(C + gh + ld * gh).x;
            }
        }
    } else if constexpr (SRC == SRC_PSI_Q) {
        const uint32_t h32 = (uint32_t)half;
#pragma unroll
        for (int k = 0; k < Cfg::E; ++k) {
            const uint32_t g = slot_gidx<Cfg, A0>(base, rs, k);
            const float2 u = __ldg(psi + g);
            const float2 w = __ldg(psi + (g | h32));
            const R ux = u.x, uy = u.y, wx = w.x, wy = w.y;
            v[k].x = fma(ux, ux, uy * uy);
            v[k].y = fma(wx, wx, wy * wy);
        }
    } else if constexpr (Cfg::LO == 0) {
        // contiguous tile (lo_g = 0): one base plus compile-time offsets
        const C2 *src = reinterpret_cast<const C2 *>(a.src) + (size_t)slot * (size_t)a.slot_elems + gbase +
                        Cfg::elem(t, 0, A0);
#pragma unroll
        for (int k = 0; k < Cfg::E; ++k) v[k] = src[(uint32_t)k << A0];
    } else {
        const C2 *src = reinterpret_cast<const C2 *>(a.src) + (size_t)slot * (size_t)a.slot_elems;
#pragma unroll
        for (int k = 0; k < Cfg::E; ++k) v[k] = src[slot_gidx<Cfg, A0>(base, rs, k)];
    }
}

// The two Pauli expectations a transformed element H(z') yields:
// c(z0) and c(z1), z0 = z' with 0 inserted at bit j, z1 = z0 | 2^j (signed).
template <typename R, typename C2>
__device__ __forceinline__ void family_pair(unsigned long long x, int j, R s, C2 h, unsigned long long zp,
                                            unsigned long long &z0, unsigned long long &z1, R &c0, R &c1) {
    z0 = insert0(zp, j);
    z1 = z0 | (1ULL << j);
    if (x) {
        const R sc = (R)2 * s;
        const int k0 = __popcll(x & z0);
        const R re = sc * h.x, im = sc * h.y;
        c0 = (R)sgn_phase(k0) * ((k0 & 1) ? im : re);
        c1 = (R)sgn_phase(k0 + 1) * ((k0 & 1) ? re : im);
    } else {
        c0 = s * (h.x + h.y);
        c1 = s * (h.x - h.y);
    }
}

// log2 on the MUFU unit, subnormal inputs flushed (callers keep x >= FLT_MIN)
__device__ __forceinline__ float lg2_ftz(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Fused moment sums of Algorithm 1 over one thread's E transformed elements:
// c = sc * h (a pair of Pauli expectations), q = c^2, and packed running
// sums of q, q^2, q^3 and q log2 q. FLT_MIN is added inside the log only:
// it leaves every q >= 2^-102 unchanged and makes q = 0 contribute 0.
// SWAP orders each pair so that c(z0) comes first (bit k of pm set: swap);
// CAND keeps the running maximum of q for the nullity candidates.
template <int E, bool SWAP, bool CAND>
__device__ __forceinline__ void moment_sums(const float2 (&h)[E], float2 sc, uint32_t pm, float2 &s2, float2 &s4,
                                            float2 &s6, float2 &sl, float &qmax) {
    const float2 tiny = make_float2(1.17549435e-38f, 1.17549435e-38f);
#pragma unroll
    for (int k = 0; k < E; ++k) {
        float2 c = mul2(sc, h[k]);
        if constexpr (SWAP) {
            if ((pm >> k) & 1u) c = make_float2(c.y, c.x);
        }
        const float2 q = mul2(c, c);
        const float2 q2 = mul2(q, q);
        s2 = add2(s2, q);
        s4 = add2(s4, q2);
        s6 = fma2(q2, q, s6);
        const float2 qt = add2(q, tiny);
        sl = fma2(q, make_float2(lg2_ftz(qt.x), lg2_ftz(qt.y)), sl);
        if constexpr (CAND) qmax = fmaxf(qmax, fmaxf(q.x, q.y));
    }
}

// Weights of the 2^ZR_FINE-z ranges of a last-pass tile (slot bits are z'
// bits 0 .. RB-1 and thread t holds z' = zb + k, so L consecutive lanes span
// L E consecutive z'). With j >= ZR_FINE (or x = 0, pair (z', z' + d/2)) the
// c(z0) of 2^ZR_FINE consecutive z' fill one range and their c(z1) another,
// s2 being ordered (c(z0)^2, c(z1)^2); with j < ZR_FINE, 2^(ZR_FINE-1) z'
// yield both c of 2^ZR_FINE consecutive z. A range spans 2^ZR_FINE / E (split)
// or 2^(ZR_FINE-1) / E lanes: within a warp its sum is written by one lane;
// across two warps (E = 16, split) both add into the zeroed row, and the sum
// of two FP32 terms does not depend on their order.
template <int E>
__device__ __forceinline__ void fine_range_weights(float2 s2, unsigned long long x, int j, unsigned long long half,
                                                   uint32_t zb, float *row, bool active) {
    static_assert(E == 32 || E == 16, "16 or 32 points per thread");
    const int lane = threadIdx.x & 31;
    const bool split = (x == 0) || (j >= ZR_FINE);
    unsigned long long z0, z1;
    if (x) {
        z0 = insert0((unsigned long long)zb, j);
        z1 = z0 | (1ULL << j);
    } else {
        z0 = zb;
        z1 = (unsigned long long)zb | half;
    }
    float wa = split ? s2.x : s2.x + s2.y, wb = s2.y;
    constexpr int LS = (1 << ZR_FINE) / E;          // lanes of a range when split (32 or 64)
    constexpr int LN = (1 << (ZR_FINE - 1)) / E;    // lanes of a range otherwise (16 or 32)
#pragma unroll
    for (int o = 1; o < LN; o <<= 1) {
        wa += __shfl_xor_sync(0xffffffffu, wa, o);
        wb += __shfl_xor_sync(0xffffffffu, wb, o);
    }
    if (split) {
        if constexpr (LS > LN) {
            if constexpr (LN < 32) {
                wa += __shfl_xor_sync(0xffffffffu, wa, LN);
                wb += __shfl_xor_sync(0xffffffffu, wb, LN);
            }
        }
        if (active && lane == 0) {
            if constexpr (LS > 32) {
                atomicAdd(row + (z0 >> ZR_FINE), wa);
                atomicAdd(row + (z1 >> ZR_FINE), wb);
            } else {
                row[z0 >> ZR_FINE] = wa;
                row[z1 >> ZR_FINE] = wb;
            }
        }
    } else if (active && (lane & (LN - 1)) == 0) {
        row[z0 >> ZR_FINE] = wa;
    }
}

// true when the range rows of a last pass with E points per thread must be
// zeroed before it (two warps add into each range)
__host__ __device__ constexpr bool ranges_accumulate(int E) { return (1 << ZR_FINE) / E > 32; }

// Families a CTA of a psi-reading strided pass transforms in turn, on the
// same tile: fewer, longer CTAs (their L1 hit rate stays near zero; N = 24:
// 2.79 ms per 128-family launch with 4 families per CTA, 2.83 with 2, 2.97
// with 1; 8 gains nothing over 4).
#ifndef SRE_STRIDED_FPC
#define SRE_STRIDED_FPC 4
#endif
template <class Cfg, int SRC> struct FamPerCta {
    static constexpr int v = (SRC == SRC_PSI_FAMILY && Cfg::G == 1 && Cfg::LO > 0) ? SRE_STRIDED_FPC : 1;
};

// One tile of one family (the rep-th family of the CTA); false when the CTA
// has no rep-th family.
// The tile of the CTA's rep-th family (one family per group when G > 1) in
// the launch's grid: (slot of group 0, tile), or false when the CTA has no
// rep-th family.
template <class Cfg, int SRC>
__device__ __forceinline__ bool pass_grid_item(const PassArgs &a, int rep, long long &slot0,
                                               unsigned long long &tile) {
    if constexpr (Cfg::G > 1) {
        slot0 = (long long)blockIdx.x * Cfg::G;
        tile = 0;
    } else if (a.fam_fast) {
        constexpr int FPC = FamPerCta<Cfg, SRC>::v;
        const unsigned long long L = blockIdx.x;
        const unsigned long long np = ((unsigned long long)a.n_fam + FPC - 1) / FPC;
        slot0 = (long long)(L % np) * FPC + rep;
        tile = L / np;
        if (rep > 0 && slot0 >= a.n_fam) return false;
    } else {
        slot0 = (long long)blockIdx.y + 65535LL * (long long)blockIdx.z;
        tile = blockIdx.x;
    }
    return true;
}

// One tile of the families slot0 + grp (grp < G) of a launch.
template <class Cfg, int SRC, int DST, int PREC>
__device__ __forceinline__ void fwht_pass_body(const PassArgs &a, long long slot0, unsigned long long tile) {
    typedef typename Cfg::Real R;
    typedef typename Cfg::C2 C2;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2 *sm = reinterpret_cast<C2 *>(smraw);
    constexpr size_t TILE_SMEM = (Cfg::NR > 1 || PREC != 0) ? sizeof(C2) * (size_t)Cfg::G * Cfg::PSIZE : 0;
    double *red = reinterpret_cast<double *>(smraw + TILE_SMEM);

    const uint32_t tid = threadIdx.x;
    const uint32_t grp = tid >> Cfg::TB;
    const uint32_t t = tid & (Cfg::T - 1);

    long long slot = slot0 + (Cfg::G > 1 ? (long long)grp : 0LL);
    const bool active = slot < a.n_fam;
    if (!active) slot = a.n_fam - 1;   // run on valid data, write nothing

    const int N = a.N;
    const int n = a.n;
    const unsigned long long dmask = (N >= 64) ? ~0ULL : ((1ULL << N) - 1ULL);
    unsigned long long x = 0, F = 0;
    if constexpr (SRC == SRC_PSI_FAMILY || DST == DST_MOMENTS || DST == DST_SPECTRUM || DST == DST_NULLCOUNT ||
                  DST == DST_CANDLIST) {
        F = a.xs ? a.xs[a.fam_base + slot] : (unsigned long long)(a.fam_base + slot);
        x = F & dmask;
    }
    const float2 *psi = a.psi;        // per-state psi / s in multi-state launches
    const double *s_ptr = a.s_ptr;
    if (a.psi_list) {
        const unsigned long long st = F >> N;
        psi = a.psi_list[st];
        s_ptr = a.s_list + st;
    }
    const int j = x ? 63 - __clzll((long long)x) : n;
    const unsigned long long half = 1ULL << n;

    // global packed index of tile element e
    const int cb_bits = a.lo_g - Cfg::LO;
    const unsigned long long cb = tile & ((1ULL << cb_bits) - 1ULL);
    const unsigned long long outer = tile >> cb_bits;
    const unsigned long long gbase = (outer << (a.lo_g + Cfg::K)) | (cb << Cfg::LO);
    auto gidx = [&](uint32_t e) -> unsigned long long {
        return gbase | ((unsigned long long)(e >> Cfg::LO) << a.lo_g) | (e & ((1u << Cfg::LO) - 1u));
    };

    C2 v[Cfg::E];
    constexpr int AL = Maps<Cfg>::last;

    // The moments epilogue wants s in FP32 in every thread; one conversion per
    // group, passed through shared memory (the transform's barriers order it).
    constexpr bool S_SHARED = DST == DST_MOMENTS && Cfg::T >= 32;
    float *s_sh = reinterpret_cast<float *>(red) + 8 * (Cfg::NT / 32);
    if constexpr (S_SHARED) {
        if (t == 0) s_sh[grp] = (float)(*s_ptr);
        if constexpr (Cfg::NR <= 1 && PREC == 0) __syncthreads();
    }

    // ---------------------------------------------------------- prologue
    pass_prologue<Cfg, SRC>(v, a, psi, slot, x, j, half, gbase, t);

    // --------------------------------------------------------- transform
    if constexpr (PREC == 0) tile_transform<Cfg>(v, sm, t, grp);
    else tc_tile_transform<Cfg, PREC>(v, sm, t, grp);

    // ---------------------------------------------------------- epilogue
    if constexpr (DST == DST_BUF) {
        if (active) {
            C2 *dst = reinterpret_cast<C2 *>(a.dst) + (size_t)slot * (size_t)a.slot_elems;
            const uint32_t base = thread_gidx<Cfg>(gbase, a.lo_g, Cfg::elem(t, 0, AL));
            const uint32_t rs = 1u << a.lo_g;
#pragma unroll
            for (int k = 0; k < Cfg::E; ++k) dst[slot_gidx<Cfg, AL>(base, rs, k)] = v[k];
        }
    } else if constexpr (DST == DST_SQMAP) {
        if (active) {
            const R s = (R)(*a.s_ptr);
            const R s2 = s * s;
            C2 *dst = reinterpret_cast<C2 *>(a.dst);
#pragma unroll
            for (int k = 0; k < Cfg::E; ++k) {
                const R p = v[k].x + v[k].y, m = v[k].x - v[k].y;
                C2 o;
                o.x = s2 * (p * p);
                o.y = s2 * (m * m);
                dst[gidx(Cfg::elem(t, k, AL))] = o;
            }
        }
    } else if constexpr (DST == DST_P) {
        if (active) {
            const R invd = (R)1 / (R)(2.0 * (double)half);
#pragma unroll
            for (int k = 0; k < Cfg::E; ++k) {
                const unsigned long long g = gidx(Cfg::elem(t, k, AL));
                a.p_out[g] = (double)((v[k].x + v[k].y) * invd);
                a.p_out[g | half] = (double)((v[k].x - v[k].y) * invd);
            }
        }
    } else if constexpr (DST == DST_SPECTRUM) {
        if (active) {
            const R s = (R)(*s_ptr);
            R *out = reinterpret_cast<R *>(a.spec_out) + (size_t)slot * (size_t)(2 * half);
#pragma unroll
            for (int k = 0; k < Cfg::E; ++k) {
                unsigned long long z0, z1;
                R c0, c1;
                family_pair<R, C2>(x, j, s, v[k], gidx(Cfg::elem(t, k, AL)), z0, z1, c0, c1);
                out[z0] = c0;
                out[z1] = c1;
            }
        }
    } else if constexpr (DST == DST_CANDLIST) {
        // every packed z' of a flagged family whose pair (c(z0), c(z1))
        // holds a |c| above the candidate threshold: counted, and listed
        // while the slot's list has room
        if (active) {
            const R s = (R)(*s_ptr);
            const R thr2 = (R)a.cand_thr * (R)a.cand_thr;
#pragma unroll
            for (int k = 0; k < Cfg::E; ++k) {
                R c0, c1;
                if (x) { c0 = (R)2 * s * v[k].x; c1 = (R)2 * s * v[k].y; }
                else { c0 = s * (v[k].x + v[k].y); c1 = s * (v[k].x - v[k].y); }
                if (c0 * c0 > thr2 || c1 * c1 > thr2) {
                    const unsigned i = atomicAdd(a.cand_cnt + slot, 1u);
                    if (i < (unsigned)a.cand_max)
                        a.cand_z[(size_t)slot * (size_t)a.cand_max + i] = (unsigned)gidx(Cfg::elem(t, k, AL));
                }
            }
        }
    } else if constexpr (DST == DST_NULLCOUNT) {
        const R s = (R)(*s_ptr);
        const R sc = x ? (R)2 * s : s;
        double cnt = 0.0;
#pragma unroll
        for (int k = 0; k < Cfg::E; ++k) {
            R c0, c1;
            if (x) { c0 = sc * v[k].x; c1 = sc * v[k].y; }
            else { c0 = s * (v[k].x + v[k].y); c1 = s * (v[k].x - v[k].y); }
            cnt += (fabs(fabs((double)c0) - 1.0) < a.eps) ? 1.0 : 0.0;
            cnt += (fabs(fabs((double)c1) - 1.0) < a.eps) ? 1.0 : 0.0;
        }
        cnt = group_sum<Cfg::T, Cfg::NT>(cnt, red);
        if (active && t == 0 && cnt > 0.0) atomicAdd(a.count_out + slot, (unsigned long long)cnt);
    } else if constexpr (DST == DST_MOMENTS) {
        static_assert(Cfg::LO == 0 && AL == 0, "moments epilogue runs on last-pass tiles");
        // z' = zb | k for slot k (last mapping: slot bits are the low RB bits).
        // q = (c(z0)^2, c(z1)^2) up to the order fixed by the parity, kept as
        // a packed pair: moments only need the unordered pair. The z-range
        // weights are read off the packed sum of q: a tile spans two ranges
        // of 2^M consecutive z (range A, then range B).
        float s;
        if constexpr (S_SHARED) s = s_sh[grp];
        else s = (float)(*s_ptr);
        const uint32_t zb = (uint32_t)gbase | Cfg::elem(t, 0, 0);
        float2 s2 = make_float2(0.f, 0.f), s4 = s2, s6 = s2, sl = s2, w = s2;
        float qmax = 0.f;
        const bool wr = a.want_ranges, cand = a.want_cand;
        // ranges of 2^ZR_FINE z (written per warp) or tile halves (2^M z)
        constexpr bool FINE = SRC == SRC_BUF && Cfg::M > ZR_FINE;
        constexpr int RLS = FINE ? ZR_FINE : Cfg::M;
        if (x) {
            const float2 sc = make_float2(2.0f * s, 2.0f * s);
            if (wr && j >= RLS) {
                // every c(z0) and every c(z1) of a range block lie in ranges
                // of their own: order each pair as (c(z0)^2, c(z1)^2) and s2
                // is the pair of weights. Bit k of pm: parity of |x & z0| for
                // z' = zb | k (z0 then carries the Im part).
                const uint32_t xd = (uint32_t)((x & ((1ULL << j) - 1ULL)) | ((x >> (j + 1)) << j));
                const uint32_t pm = walsh_mask5(xd & (Cfg::E - 1)) ^ ((__popc(xd & zb) & 1) ? 0xFFFFFFFFu : 0u);
                if (cand) moment_sums<Cfg::E, true, true>(v, sc, pm, s2, s4, s6, sl, qmax);
                else moment_sums<Cfg::E, true, false>(v, sc, pm, s2, s4, s6, sl, qmax);
                w = s2;
            } else {
                if (cand) moment_sums<Cfg::E, false, true>(v, sc, 0u, s2, s4, s6, sl, qmax);
                else moment_sums<Cfg::E, false, false>(v, sc, 0u, s2, s4, s6, sl, qmax);
                if (wr && !FINE) {
                    // both c of a pair lie in the range picked by bit M-1 of z'
                    constexpr int RBIT = Cfg::M > 0 ? Cfg::M - 1 : 0;
                    if constexpr (RBIT >= Cfg::RB) {
                        const float all = s2.x + s2.y;
                        w = ((zb >> RBIT) & 1u) ? make_float2(0.f, all) : make_float2(all, 0.f);
                    } else {
                        // tiles of at most 2 RB bits: the range bit is a slot bit
#pragma unroll
                        for (int k = 0; k < Cfg::E; ++k) {
                            const float2 c = mul2(sc, v[k]);
                            const float qq = c.x * c.x + c.y * c.y;
                            if ((k >> RBIT) & 1) w.y += qq;
                            else w.x += qq;
                        }
                    }
                }
            }
        } else {
            const float2 sc = make_float2(s, s);
            typename Cfg::C2 hs[Cfg::E];
#pragma unroll
            for (int k = 0; k < Cfg::E; ++k) hs[k] = make_float2(v[k].x + v[k].y, v[k].x - v[k].y);
            if (cand) moment_sums<Cfg::E, false, true>(hs, sc, 0u, s2, s4, s6, sl, qmax);
            else moment_sums<Cfg::E, false, false>(hs, sc, 0u, s2, s4, s6, sl, qmax);
            w = s2;                    // z' -> range A, z' + d/2 -> range B
        }
        if constexpr (FINE) {
            if (wr) fine_range_weights<Cfg::E>(s2, x, j, half, zb, a.rw_out + (size_t)slot * (size_t)a.rw_stride, active);
        }
        float acc[6] = {s2.x + s2.y, s4.x + s4.y, s6.x + s6.y, sl.x + sl.y, w.x, w.y};
        double out[6];
        float omx;
        group_reduce<Cfg::T, Cfg::NT, 6>(acc, qmax, out, omx, red);
        if (active && t == 0 && a.fam_out) {
            FamMoments &o = a.fam_out[a.fam_base + slot];
            o.m[0] = out[0]; o.m[1] = out[1]; o.m[2] = out[2]; o.m[3] = out[3];
            o.cand = (cand && omx > a.cand_thr * a.cand_thr) ? 1ull : 0ull;
        } else if (active && t == 0) {
            const long long tiles = (long long)(half >> Cfg::M) > 0 ? (long long)(half >> Cfg::M) : 1;
            TilePartial &tp = a.tile_out[(size_t)slot * (size_t)tiles + tile];
            tp.m[0] = out[0]; tp.m[1] = out[1]; tp.m[2] = out[2]; tp.m[3] = out[3];
            tp.w[0] = out[4]; tp.w[1] = out[5];
            tp.cand = (cand && omx > a.cand_thr * a.cand_thr) ? 1u : 0u;
        }
    }
}

template <class Cfg, int SRC, int DST, int PREC = 0>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB) fwht_pass_kernel(const PassArgs a) {
    constexpr int FPC = FamPerCta<Cfg, SRC>::v;
    long long slot0;
    unsigned long long tile;
    if constexpr (FPC == 1) {
        pass_grid_item<Cfg, SRC>(a, 0, slot0, tile);
        fwht_pass_body<Cfg, SRC, DST, PREC>(a, slot0, tile);
    } else {
        if (!a.fam_fast) {
            pass_grid_item<Cfg, SRC>(a, 0, slot0, tile);
            fwht_pass_body<Cfg, SRC, DST, PREC>(a, slot0, tile);
            return;
        }
#pragma unroll 1
        for (int r = 0; r < FPC; ++r) {
            if (r) __syncthreads();                 // the tile buffer is reused
            if (!pass_grid_item<Cfg, SRC>(a, r, slot0, tile)) break;
            fwht_pass_body<Cfg, SRC, DST, PREC>(a, slot0, tile);
        }
    }
}


template <class Cfg, int SRC, int DST, int PREC = 0>
cudaError_t launch_cfg(const PassArgs &a, int tiles, cudaStream_t st) {
    const size_t tile_smem = (Cfg::NR > 1 || PREC != 0) ? sizeof(typename Cfg::C2) * (size_t)Cfg::G * Cfg::PSIZE : 0;
    const size_t smem = tile_smem + sizeof(double) * (8 * (Cfg::NT / 32) + 8);
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(fwht_pass_kernel<Cfg, SRC, DST, PREC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid;
    PassArgs b = a;
    b.fam_fast = 0;
    if constexpr (Cfg::G > 1) {
        grid = dim3((unsigned)((a.n_fam + Cfg::G - 1) / Cfg::G), 1, 1);
    } else {
        const long long nf = a.n_fam;
        const long long total = nf * (long long)tiles;
        if ((SRC == SRC_PSI_FAMILY || SRC == SRC_PSI_Q) && nf > 1 && tiles > 1 &&
            total < 0x7fffffffLL) {
            constexpr int FPC = FamPerCta<Cfg, SRC>::v;
            b.fam_fast = 1;
            grid = dim3((unsigned)(((nf + FPC - 1) / FPC) * (long long)tiles), 1, 1);
        } else {
            grid = dim3((unsigned)tiles, (unsigned)(nf < 65535 ? nf : 65535), (unsigned)((nf + 65534) / 65535));
        }
    }
    fwht_pass_kernel<Cfg, SRC, DST, PREC><<<grid, Cfg::NT, smem, st>>>(b);
    return cudaGetLastError();
}

} // namespace sre
