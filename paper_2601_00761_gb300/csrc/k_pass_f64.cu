// Instantiations: FP64 passes (nullity recheck, x-marginal, FP64 spectra).
#include "k_pass_dispatch.cuh"
namespace sre {
cudaError_t launch_f64_single(int M, int src, int dst, const PassArgs &a, cudaStream_t st) {
    switch (M) {
#define C(m) case m: return launch_sd<KIND_SINGLE, SingleCfgOf<double, m>::type>(src, dst, a, 1, st);
    C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12)
#undef C
    default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_f64_strided(int K, int src, int dst, const PassArgs &a, int tiles, cudaStream_t st) {
    switch (K) {
#define C(k) case k: return launch_sd<KIND_STRIDED, TileCfg<double, F64_STRIDED_M, F64_STRIDED_M - k, 4, 1>>(src, dst, a, tiles, st);
    C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9)
#undef C
    default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_f64_row(int M, int src, int dst, const PassArgs &a, int tiles, cudaStream_t st) {
    if (M != F64_ROW_M) return cudaErrorInvalidValue;
    return launch_sd<KIND_ROW, TileCfg<double, F64_ROW_M, 0, 4, 1>>(src, dst, a, tiles, st);
}
} // namespace sre
