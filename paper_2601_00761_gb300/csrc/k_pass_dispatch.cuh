// k_pass_dispatch.cuh -- (source, destination) combinations each tile
// geometry is instantiated for, shared by the k_pass_*.cu units.
#pragma once
#include <type_traits>
#include "k_pass.cuh"

namespace sre {

enum PassKind { KIND_SINGLE = 0, KIND_STRIDED = 1, KIND_ROW = 2 };

#define SRE_ALLOW(R, KIND, SRC, DST) \
    template <int M, int LO, int RB, int G> struct AllowedK<R, KIND, SRC, DST, M, LO, RB, G> { static constexpr bool value = true; };

template <typename R, int KIND, int SRC, int DST, int M, int LO, int RB, int G>
struct AllowedK { static constexpr bool value = false; };

SRE_ALLOW(float, KIND_SINGLE, SRC_PSI_FAMILY, DST_MOMENTS)
SRE_ALLOW(float, KIND_SINGLE, SRC_PSI_FAMILY, DST_SPECTRUM)
SRE_ALLOW(float, KIND_SINGLE, SRC_GRAM, DST_MOMENTS)
SRE_ALLOW(float, KIND_SINGLE, SRC_GRAM, DST_SPECTRUM)
SRE_ALLOW(float, KIND_STRIDED, SRC_PSI_FAMILY, DST_BUF)
SRE_ALLOW(float, KIND_STRIDED, SRC_BUF, DST_BUF)
SRE_ALLOW(float, KIND_ROW, SRC_BUF, DST_MOMENTS)
SRE_ALLOW(float, KIND_ROW, SRC_BUF, DST_SPECTRUM)
SRE_ALLOW(float, KIND_SINGLE, SRC_PSI_FAMILY, DST_CANDLIST)
SRE_ALLOW(float, KIND_ROW, SRC_BUF, DST_CANDLIST)
SRE_ALLOW(double, KIND_SINGLE, SRC_PSI_FAMILY, DST_NULLCOUNT)
SRE_ALLOW(double, KIND_SINGLE, SRC_PSI_FAMILY, DST_SPECTRUM)
SRE_ALLOW(double, KIND_SINGLE, SRC_PSI_Q, DST_SQMAP)
SRE_ALLOW(double, KIND_SINGLE, SRC_BUF, DST_P)
SRE_ALLOW(double, KIND_STRIDED, SRC_PSI_FAMILY, DST_BUF)
SRE_ALLOW(double, KIND_STRIDED, SRC_PSI_Q, DST_BUF)
SRE_ALLOW(double, KIND_STRIDED, SRC_BUF, DST_BUF)
SRE_ALLOW(double, KIND_ROW, SRC_BUF, DST_NULLCOUNT)
SRE_ALLOW(double, KIND_ROW, SRC_BUF, DST_SPECTRUM)
SRE_ALLOW(double, KIND_ROW, SRC_BUF, DST_SQMAP)
SRE_ALLOW(double, KIND_ROW, SRC_BUF, DST_P)
#undef SRE_ALLOW

// Tensor-core variants exist for FP32 tiles whose groups are whole warps.
template <class Cfg> struct TcOK {
    static constexpr bool value = std::is_same<typename Cfg::Real, float>::value && Cfg::T >= 32;
};

template <int KIND, class Cfg, int SRC, int DST>
cudaError_t launch_if(const PassArgs &a, int tiles, cudaStream_t st) {
    if constexpr (DST == DST_CANDLIST && AllowedK<typename Cfg::Real, KIND, SRC, DST, Cfg::M, Cfg::LO, Cfg::RB, Cfg::G>::value) {
        return launch_cfg<Cfg, SRC, DST, 0>(a, tiles, st);   // FP32 butterflies whatever the sweep's precision
    } else if constexpr (AllowedK<typename Cfg::Real, KIND, SRC, DST, Cfg::M, Cfg::LO, Cfg::RB, Cfg::G>::value) {
        if (a.precision == 0) return launch_cfg<Cfg, SRC, DST, 0>(a, tiles, st);
        if constexpr (TcOK<Cfg>::value) {
            if (a.precision == 2) return launch_cfg<Cfg, SRC, DST, 2>(a, tiles, st);
            if (a.precision == 3) return launch_cfg<Cfg, SRC, DST, 3>(a, tiles, st);
        } else {
            return launch_cfg<Cfg, SRC, DST, 0>(a, tiles, st);   // tiles below one warp: FP32 butterflies
        }
        return cudaErrorInvalidValue;
    } else {
        return cudaErrorInvalidValue;
    }
}

template <int KIND, class Cfg>
cudaError_t launch_sd(int src, int dst, const PassArgs &a, int tiles, cudaStream_t st) {
#define SRE_D(S)                                                                 \
    switch (dst) {                                                               \
    case DST_BUF: return launch_if<KIND, Cfg, S, DST_BUF>(a, tiles, st);         \
    case DST_MOMENTS: return launch_if<KIND, Cfg, S, DST_MOMENTS>(a, tiles, st); \
    case DST_SPECTRUM: return launch_if<KIND, Cfg, S, DST_SPECTRUM>(a, tiles, st); \
    case DST_NULLCOUNT: return launch_if<KIND, Cfg, S, DST_NULLCOUNT>(a, tiles, st); \
    case DST_SQMAP: return launch_if<KIND, Cfg, S, DST_SQMAP>(a, tiles, st);     \
    case DST_P: return launch_if<KIND, Cfg, S, DST_P>(a, tiles, st);             \
    case DST_CANDLIST: return launch_if<KIND, Cfg, S, DST_CANDLIST>(a, tiles, st); \
    default: return cudaErrorInvalidValue;                                       \
    }
    switch (src) {
    case SRC_PSI_FAMILY: SRE_D(SRC_PSI_FAMILY)
    case SRC_PSI_Q: SRE_D(SRC_PSI_Q)
    case SRC_BUF: SRE_D(SRC_BUF)
    case SRC_GRAM: SRE_D(SRC_GRAM)
    default: return cudaErrorInvalidValue;
    }
#undef SRE_D
}

// Geometry of the single-pass tile of M bits: RB register bits, G families per CTA.
template <typename R> struct SingleRB;
template <> struct SingleRB<float> { static constexpr int v = 5; };
template <> struct SingleRB<double> { static constexpr int v = 4; };

template <typename R, int M>
struct SingleCfgOf {
    static constexpr int RB = M < SingleRB<R>::v ? M : SingleRB<R>::v;
    static constexpr int TB = M - RB;
    static constexpr int G = TB >= 8 ? 1 : (256 >> TB);
    typedef TileCfg<R, M, 0, RB, G> type;
};

cudaError_t launch_f32_single(int M, int src, int dst, const PassArgs &a, cudaStream_t st);
cudaError_t launch_f32_strided(int MS, int K, int src, int dst, const PassArgs &a, int tiles, cudaStream_t st);
cudaError_t launch_f32_row(int M, int src, int dst, const PassArgs &a, int tiles, cudaStream_t st);
cudaError_t launch_f64_single(int M, int src, int dst, const PassArgs &a, cudaStream_t st);
cudaError_t launch_f64_strided(int K, int src, int dst, const PassArgs &a, int tiles, cudaStream_t st);
cudaError_t launch_f64_row(int M, int src, int dst, const PassArgs &a, int tiles, cudaStream_t st);

// strided tile: 2^K rows x 2^(MS-K) columns; FP32 MS = 13 for every K (64 KB,
// at least 8 columns = 64 contiguous bytes per row, two CTAs per SM so one
// CTA's loads overlap the other's butterflies); FP64 MS = 13 (128 KB)
constexpr int F32_STRIDED_KMAX = 10, F32_ROW_MMIN = 10, F32_ROW_MMAX = 14, F32_SINGLE_MMAX = 14;
// register bits of the 13-bit FP32 row pass: 4 (512 threads x 16 points, two
// CTAs per SM: 32 warps) or 5 (256 x 32)
#ifndef SRE_ROW13_RB
#define SRE_ROW13_RB 5
#endif
constexpr int F32_ROW13_RB = SRE_ROW13_RB;
// register bits of the 10-row strided FP32 pass (2^10 rows x 8 columns):
// 5 (256 threads x 32 points) or 4 (512 threads x 16 points)
#ifndef SRE_STRIDED10_RB
#define SRE_STRIDED10_RB 5
#endif
constexpr int F32_STRIDED10_RB = SRE_STRIDED10_RB;
// whether the FP32 row pass of M bits accumulates its z-range weights (the
// caller zeroes the rows first)
constexpr bool f32_row_ranges_accumulate(int M) { return ranges_accumulate(1 << (M == 13 ? F32_ROW13_RB : 5)); }
__host__ __device__ constexpr int f32_strided_ms(int K) { return K + 3 > 13 ? K + 3 : 13; }
constexpr int F64_STRIDED_M = 13, F64_STRIDED_KMAX = 9, F64_ROW_M = 12, F64_SINGLE_MMAX = 12;

} // namespace sre
