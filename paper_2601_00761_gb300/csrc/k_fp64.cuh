// k_fp64.cuh -- FP64 helpers: exact widening of FP32 data, compensated sums.
#pragma once

#include <cuda_runtime.h>

namespace sre {

// binary32 -> binary64 by re-packing the fields (exact: every float is a
// double). The conversion instruction runs on the FP64 pipe, which issues
// one warp instruction per 16 cycles on this part; normal numbers and zeros
// go through integer operations instead, and only subnormals, inf and NaN
// take the instruction.
__device__ __forceinline__ double f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu, sg = u & 0x80000000u;
    if (e == 0u && m == 0u) return __hiloint2double((int)sg, 0);
    if (e - 1u >= 254u) return (double)f;
    return __hiloint2double((int)(sg | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// Neumaier's compensated summation (Neumaier 1974, the Kahan-Babuska form):
// s is the running sum and c gathers the rounding error of every addition,
// so s + c carries a sum of many terms to about one rounding of the result.
struct NeuSum {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double x) {
        const double t = s + x;
        c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __device__ __forceinline__ double value() const { return s + c; }
};

}  // namespace sre
