// Instantiations: FP32 single-pass family transforms (whole family in one tile).
#include "k_pass_dispatch.cuh"
namespace sre {
cudaError_t launch_f32_single(int M, int src, int dst, const PassArgs &a, cudaStream_t st) {
    switch (M) {
#define C(m) case m: return launch_sd<KIND_SINGLE, SingleCfgOf<float, m>::type>(src, dst, a, 1, st);
    C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13) C(14)
#undef C
    default: return cudaErrorInvalidValue;
    }
}
} // namespace sre
