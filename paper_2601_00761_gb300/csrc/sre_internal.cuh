// sre_internal.cuh -- shared device code of the GB300 FWHT Pauli-spectrum library.
//
// The family transform (Algorithm 1, loop body; Eq. Pxz-corr) is evaluated in
// a packed form. For x != 0 let j be the highest set bit of x. The summand
// f_x(b) = conj(psi[b^x]) psi[b] obeys f_x(b^x) = conj f_x(b), so pairing b
// with b^x (b_j = 0) gives
//     F_x(z) = sum_{b: b_j=0} (-1)^{z.b} * (2 Re f_x(b)   if x.z even,
//                                          2i Im f_x(b)  if x.z odd).
// Writing b' = b with bit j deleted, the complex vector h(b') = 2 f_x(b) of
// length 2^{N-1} has the transform H(z') = A(z') + i B(z') whose real part
// gives every even-parity c and whose imaginary part every odd-parity c:
//     c_{x,z} = s (-1)^{floor((k+1)/2)} * (k even ? Re : Im) H(z'),  k = |x&z|,
// z' = z with bit j deleted. Each amplitude of psi is read once per family
// and the transform has 2^{N-1} complex points. For x = 0 (j = N-1) the
// packed vector is h(g) = (|psi[g]|^2, |psi[g + d/2]|^2) and
// c_{0,z'} = s (Re + Im) H, c_{0,z' + d/2} = s (Re - Im) H.
//
// A transform of n = N-1 bits runs as one or more passes. Each pass moves
// tiles of 2^M complex elements through shared memory; a tile is 2^K rows
// (transformed) x 2^LO columns (contiguous in global memory, not
// transformed). Inside a tile each thread holds 2^RB elements; rounds of up
// to RB butterfly stages run in registers and tiles are re-distributed
// through shared memory between rounds (one __syncthreads per round).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// CTAs per SM targeted by the register allocation of 256-thread tiles of at
// most 64 KB (a build-time tuning constant).
#ifndef SRE_MINB_SMALL
#define SRE_MINB_SMALL 2
#endif

namespace sre {

template <typename R> struct V2;
template <> struct V2<float> { typedef float2 T; };
template <> struct V2<double> { typedef double2 T; };

template <typename T>
__device__ __forceinline__ T cadd(T a, T b) { T r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T>
__device__ __forceinline__ T csub(T a, T b) { T r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

// Packed FP32x2 arithmetic of sm_100+ (one instruction per complex add;
// each lane rounds to nearest exactly as the scalar instruction does).
__device__ __forceinline__ unsigned long long f2u(float2 a) { return *reinterpret_cast<unsigned long long *>(&a); }
__device__ __forceinline__ float2 u2f(unsigned long long a) { return *reinterpret_cast<float2 *>(&a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)), "l"(f2u(c)));
    return u2f(d);
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return add2(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) { return sub2(a, b); }

__host__ __device__ __forceinline__ unsigned long long insert0(unsigned long long v, int j) {
    unsigned long long lo = v & ((1ULL << j) - 1ULL);
    return ((v >> j) << (j + 1)) | lo;
}

// bits of the device error word
constexpr int SRE_ERR_TIMEOUT = 1;      // a bounded wait ran out

// Per-tile partial sums of the last pass (FP64): c^2, c^4, c^6, c^2 log2 c^2,
// the two z-range weights the tile contributes to, and the FP32 nullity
// candidate flag (some |c| above PassArgs::cand_thr).
struct TilePartial {
    double m[4];
    double w[2];
    unsigned int cand;     // 1 if the tile holds a |c| > cand_thr
    unsigned int pad;
    double pad2;
};

// Per-family sums (FP64) and candidate count.
struct FamMoments {
    double m[4];
    unsigned long long cand;
};

// ------------------------------------------------------------------ tile
template <typename R, int M_, int LO_, int RB_, int G_>
struct TileCfg {
    typedef R Real;
    typedef typename V2<R>::T C2;
    static constexpr int M = M_;
    static constexpr int LO = LO_;
    static constexpr int RB = RB_;
    static constexpr int G = G_;
    static constexpr int TB = M - RB;
    static constexpr int T = 1 << TB;
    static constexpr int E = 1 << RB;
    static constexpr int NT = T * G;
    static constexpr int K = M - LO;
    static constexpr int NR = RB > 0 ? (K + RB - 1) / RB : 0;
    static constexpr int SIZE = 1 << M;
    // CTAs per SM the register budget is sized for: tiles of at most 64 KB
    // (FP32 M <= 13) run several per SM so load and compute phases overlap
    // (256 threads with 32 points each, or 512 threads with 16)
    static constexpr int MINB = (G == 1 && sizeof(C2) * SIZE <= 65536 && (NT == 256 || NT == 512)) ? SRE_MINB_SMALL : 1;
    static_assert(TB >= 0, "tile smaller than a thread's registers");
    static_assert(K >= 0, "bad tile");

    // transform range i covers bits [range_lo(i), range_hi(i)); rounds run i = NR-1 .. 0
    __host__ __device__ static constexpr int range_lo(int i) { return LO + i * RB; }
    __host__ __device__ static constexpr int range_hi(int i) { return (LO + (i + 1) * RB < M) ? LO + (i + 1) * RB : M; }
    // slot bits of the round for range i: [slot_base(i), slot_base(i) + RB)
    __host__ __device__ static constexpr int slot_base(int i) { return range_hi(i) - RB > 0 ? range_hi(i) - RB : 0; }

    // element index of (thread t, slot k) when the slot bits start at a;
    // elem(t, k, a) = elem(t, 0, a) ^ (k << a) (disjoint bits)
    __device__ static __forceinline__ uint32_t elem(uint32_t t, uint32_t k, int a) {
        return (t & ((1u << a) - 1u)) | (k << a) | ((t >> a) << (a + RB));
    }
    // Shared-memory layout: one padding element per 2^RB elements,
    // phys(e) = e + (e >> RB). Bank-conflict-free for every round mapping of
    // the instantiated tiles, and additive over disjoint bit fields, so
    // phys(elem(t, k, a)) = phys(elem(t, 0, a)) + phys(k << a): a round's
    // addresses are one per-thread base plus a compile-time offset per slot.
    static constexpr int PSIZE = RB > 0 ? SIZE + (SIZE >> RB) : SIZE;
    __host__ __device__ static constexpr uint32_t pad(uint32_t e) { return RB > 0 ? e + (e >> RB) : e; }
    __device__ static __forceinline__ uint32_t phys(uint32_t e, uint32_t g) { return g * (uint32_t)PSIZE + pad(e); }
};

template <typename C2, int E, int S0, int S1>
__device__ __forceinline__ void butterflies(C2 (&v)[E]) {
#pragma unroll
    for (int s = S0; s < S1; ++s) {
#pragma unroll
        for (int k = 0; k < E; ++k) {
            if (!(k & (1 << s))) {
                C2 a = v[k], b = v[k | (1 << s)];
                v[k] = cadd(a, b);
                v[k | (1 << s)] = csub(a, b);
            }
        }
    }
}

template <class Cfg, int r>
struct Rounds {
    typedef typename Cfg::C2 C2;
    static constexpr int i = Cfg::NR - 1 - r;
    static constexpr int a = Cfg::slot_base(i);
    __device__ static __forceinline__ void run(C2 (&v)[Cfg::E], C2 *sm, uint32_t t, uint32_t g) {
        C2 *pb = sm + Cfg::phys(Cfg::elem(t, 0, a), g);
        if constexpr (r > 0) {
            __syncthreads();
#pragma unroll
            for (int k = 0; k < Cfg::E; ++k) v[k] = pb[Cfg::pad((uint32_t)k << a)];
        }
        butterflies<C2, Cfg::E, Cfg::range_lo(i) - a, Cfg::range_hi(i) - a>(v);
        if constexpr (r < Cfg::NR - 1) {
#pragma unroll
            for (int k = 0; k < Cfg::E; ++k) pb[Cfg::pad((uint32_t)k << a)] = v[k];
            Rounds<Cfg, r + 1>::run(v, sm, t, g);
        }
    }
};

// Slot base of the first (top) and last (bottom) rounds: the element mapping
// in which data enters and leaves the register file.
template <class Cfg> struct Maps {
    static constexpr int first = Cfg::NR > 0 ? Cfg::slot_base(Cfg::NR - 1) : (Cfg::M - Cfg::RB > 0 ? Cfg::M - Cfg::RB : 0);
    static constexpr int last = Cfg::NR > 0 ? Cfg::slot_base(0) : first;
};

template <class Cfg>
__device__ __forceinline__ void tile_transform(typename Cfg::C2 (&v)[Cfg::E], typename Cfg::C2 *sm,
                                               uint32_t t, uint32_t g) {
    if constexpr (Cfg::NR > 0) Rounds<Cfg, 0>::run(v, sm, t, g);
}

// z-ranges of the two-level sampler: 2^ZR_FINE consecutive z per range when
// the last pass of a multi-pass plan has tiles of more than 2^ZR_FINE points;
// otherwise one range is one half of a last-pass tile (2^M z).
constexpr int ZR_FINE = 10;

// ------------------------------------------------------------- pass args
enum SrcMode { SRC_PSI_FAMILY = 0, SRC_PSI_Q = 1, SRC_BUF = 2, SRC_GRAM = 3 };
enum DstMode {
    DST_BUF = 0,        // store the partially transformed tile
    DST_MOMENTS = 1,    // family epilogue: moments, candidates, z-range weights
    DST_SPECTRUM = 2,   // write c_{x,z} for all z
    DST_NULLCOUNT = 3,  // count | |c| - 1 | < eps
    DST_SQMAP = 4,      // marginal: (Hr, Hi) -> ((Hr+Hi)^2, (Hr-Hi)^2)
    DST_P = 5,          // marginal: p[g] = (Hr+Hi)/d, p[g + d/2] = (Hr-Hi)/d
    DST_SAMPLE = 6,     // z sampler: c^2 of one z-range into shared memory
    DST_CANDLIST = 7    // nullity candidates of flagged families: packed z' lists
};

struct PassArgs {
    const float2 *psi;                 // complex64 state
    const unsigned long long *xs;      // family X-masks, or NULL: x = fam_base + slot
    long long fam_base;                // first family of the launch
    long long n_fam;                   // families in the launch
    void *src;                         // intermediate in  (slot stride: slot_elems complex)
    void *dst;                         // intermediate out
    long long slot_elems;              // 2^n
    int N, n;                          // qubits, packed bits (N - 1)
    int lo_g;                          // global bit of this pass's row stride
    int range_log2;                    // z-range size of the two-level sampler
    const double *s_ptr;               // 1 / sum |psi|^2
    TilePartial *tile_out;             // [slot][tile]
    void *spec_out;                    // c (float or double): [slot][d]
    unsigned long long *count_out;     // [slot]
    double *p_out;                     // marginal output p[d]
    double eps;                        // nullity tolerance
    float cand_thr;                    // FP32 candidate threshold
    int want_ranges;                   // DST_MOMENTS: also produce the z-range weights
    int want_cand;                     // DST_MOMENTS: also flag nullity candidates (exact sweeps)
    // DST_MOMENTS on last-pass tiles of more than 2^ZR_FINE points: the
    // weight of every 2^ZR_FINE-z range, one row of rw_stride floats per slot
    float *rw_out;
    long long rw_stride;
    // SRC_GRAM (reduced state of the low N qubits of a larger state):
    // C = Psi Psi^H, column-major with leading dimension gram_ld,
    // C[r][c] = sum_e psi(r, e) conj(psi(c, e))
    const float2 *gram;
    long long gram_ld;
    // Several states of the same N in one launch: the family index F (from xs
    // or fam_base + slot) is (state << N) | x; psi and s come from these
    // per-state device arrays. NULL for the one-state entry points.
    const float2 *const *psi_list;
    const double *s_list;
    int precision;                     // 0: FP32 butterflies; 2, 3: split-BF16 tensor cores (FP32 tiles)
    int *err_flag;                     // device error word (SRE_ERR_* bits), or NULL
    // CTA order: 0 = tile-major (blockIdx.x = tile, y/z = family); 1 = one
    // linear grid with the family fastest, so that the families in flight
    // work on the same tile at once and share its psi lines in L2.
    int fam_fast;
    // DST_CANDLIST: per slot, the number of packed z' whose pair holds a
    // |c| > cand_thr (cand_cnt, counted on past cand_max) and the first
    // cand_max of them (cand_z, [slot][cand_max], in no fixed order)
    unsigned *cand_cnt;
    unsigned *cand_z;
    int cand_max;
    // DST_MOMENTS on single-tile families: when set, the family's sums go
    // straight to fam_out[fam_base + slot] instead of a tile partial
    FamMoments *fam_out;
};


} // namespace sre
