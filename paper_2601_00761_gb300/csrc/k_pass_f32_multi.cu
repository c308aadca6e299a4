// Instantiations: FP32 strided passes (2^K rows x 2^(MS-K) columns) and row passes.
#include "k_pass_dispatch.cuh"
namespace sre {
cudaError_t launch_f32_strided(int MS, int K, int src, int dst, const PassArgs &a, int tiles, cudaStream_t st) {
    if (MS != f32_strided_ms(K)) return cudaErrorInvalidValue;
    switch (K) {
#define C(k) case k: return launch_sd<KIND_STRIDED, TileCfg<float, f32_strided_ms(k), f32_strided_ms(k) - k, (k == 10 ? F32_STRIDED10_RB : 5), 1>>(src, dst, a, tiles, st);
    C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10)
#undef C
    default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_f32_row(int M, int src, int dst, const PassArgs &a, int tiles, cudaStream_t st) {
    switch (M) {
#define C(m) case m: return launch_sd<KIND_ROW, TileCfg<float, m, 0, (m == 13 ? F32_ROW13_RB : 5), 1>>(src, dst, a, tiles, st);
    C(10) C(11) C(12) C(13) C(14)
#undef C
    default: return cudaErrorInvalidValue;
    }
}
} // namespace sre
