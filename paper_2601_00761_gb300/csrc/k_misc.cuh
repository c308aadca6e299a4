// k_misc.cuh -- declarations of the support kernels' launchers.
#pragma once
#include "sre_internal.cuh"

namespace sre {

// slots of the device scalar block
enum { SCAL_NORM2 = 0, SCAL_S = 1, SCAL_N = 8 };
constexpr int NORM_BLOCKS = 1216;          // 152 SMs x 8
constexpr unsigned long long SCAN_CHUNK = 4096;
// totals of an exact sweep (per state): sum over families of c^2, c^4, c^6,
// c^2 log2 c^2 sums, candidate count, sum over x != 0 of (sum_z c^4)^2, and
// the x = 0 family's sum_z c^4 (the last two give the fluctuation ratio r_2)
constexpr int TOT_N = 7;

struct DrawInfo {
    unsigned long long range;   // z-range (size 2^RL) of the draw
    double t;                   // target within the range, in units of c^2
    double wr;                  // the range's weight (sum of its c^2)
    double pad;
};

cudaError_t launch_norm2(const float2 *psi, int N, double *scal, double *partial, cudaStream_t st);

// FP64 recount of flagged families at their listed candidates (k_null.cu).
// Family i of the launch is xs[fam_base + i] (F = (state << N) | x when
// psi_list is set); its candidate count and list come from the FP32
// DST_CANDLIST pass. counts[i] receives the family's stabilizer count, or 0
// when it had no candidate or more than kdirect (<= cand_max, <=
// NULL_CAND_MAX) of them; in the latter case F is appended to ovf (ovf_n).
constexpr int NULL_CAND_MAX = 64;
struct NullDirectArgs {
    const float2 *psi;
    const double *s_ptr;
    const float2 *const *psi_list;
    const double *s_list;
    int N;
    const unsigned long long *xs;
    long long fam_base;
    const unsigned *cand_cnt;
    const unsigned *cand_z;
    int cand_max, kdirect;
    double eps;
    unsigned long long *counts, *ovf, *ovf_n;
};
cudaError_t launch_null_direct(const NullDirectArgs &a, long long n_fam, cudaStream_t st);
// per-family sums of a launch's tile partials into fm[fm_base + slot], or,
// with perm (processing order -> family index), into fm[perm[fam_base + slot]]
cudaError_t launch_fam_reduce(const TilePartial *tp, long long n_fam, int tiles, const unsigned long long *xs,
                              long long fam_base, int N, int M_last, int RL, FamMoments *fm, long long fm_base,
                              float *W, long long nr, cudaStream_t st, const unsigned long long *perm = nullptr);
cudaError_t launch_exact_totals(const FamMoments *fm, long long n_fam, double *partial, int n_part,
                                double *out, unsigned long long *flag_list, unsigned long long *n_flag,
                                cudaStream_t st);
cudaError_t launch_sum_u64(const unsigned long long *v, long long n, unsigned long long *out, cudaStream_t st);
cudaError_t launch_scan(const double *p, unsigned long long n, double *cdf, double *bsum, cudaStream_t st);
cudaError_t launch_draw_x(const double *cdf, int N, long long n_x, int mode, unsigned long long seed,
                          unsigned long long ctr0, unsigned long long *xs, cudaStream_t st);
cudaError_t launch_zrange_select(const float *Wf, long long nr, long long n_fam, long long fam_base, int z_per_x,
                                 unsigned long long seed, unsigned long long ctr0, DrawInfo *draws,
                                 const unsigned long long *perm, cudaStream_t st);
cudaError_t launch_mc_stats(const FamMoments *fm, const float *cz, long long n_x, int z_per_x, int N, int mode,
                            double *y, double *out, cudaStream_t st);
cudaError_t launch_norm2_multi(const float2 *const *psi_list, int n_states, int N, double *partial, int nb,
                               double *norm2, double *s, cudaStream_t st);
cudaError_t launch_state_totals(const FamMoments *fm, long long fm_first_family, int N, int s0, int ns,
                                double *totals, unsigned long long *flags, unsigned long long *n_flag,
                                cudaStream_t st);
cudaError_t launch_count_scatter(const unsigned long long *flags, const unsigned long long *counts, long long n,
                                 int N, unsigned long long *state_count, cudaStream_t st);
cudaError_t launch_philox_test(const unsigned long long *ctr_key, unsigned long long *out, int n, cudaStream_t st);

// z sampler (k_sample.cu): recompute the c of each draw's range and pick z by
// the exact fixed-point scan of c^2 over the range. fine: ranges of 2^ZR_FINE z
// recomputed from the folded last-pass tile; else a range is a tile half.
// one warp whose mbarrier wait can only end by its bound (k_sample.cu);
// src16: 16 readable, 16-byte aligned device bytes; err: device word
cudaError_t launch_wait_selftest(const void *src16, int *err, cudaStream_t st);
// z draws of a launch's families (k_sample.cu); perm as for launch_fam_reduce
cudaError_t launch_zsample(int single, int fine, int M, const PassArgs &a, const DrawInfo *draws, int z_per_x,
                           unsigned long long *zs, float *cz, const unsigned long long *perm, cudaStream_t st);

// gates (k_gates.cu)
struct GateRow { unsigned char op, q0, q1; };
constexpr unsigned char GATE_OP_U2 = 6;   // general two-qubit gate (matrix table indexed by row)
constexpr int GATE_BLOCK_MAX_U2 = 512;     // two-qubit matrices per block (64 KB of shared memory)
cudaError_t launch_gate_blocks(float2 *psi, int N, const GateRow *gates_dev, const float2 *mats_dev,
                               const int *blocks_host, int n_blocks, const unsigned char *block_qubits_host,
                               cudaStream_t st);
constexpr int GATE_BLOCK_Q = 13;   // qubits per fused gate block (2^13 amplitudes, 64 KB of shared memory)
constexpr int GATE_BLOCK_LOW = 5;  // qubits 0..4 always in the block (256-byte contiguous runs)

// tcgen05 self-test GEMM (k_tc05.cu): D = A B^T, BF16 in, FP32 out
cudaError_t launch_tc05_gemm_selftest(const void *A, const void *B, float *D, int M, int N, int K, int swizzle,
                                      int *err, cudaStream_t st);

// Gram matrix C = Psi Psi^H of the reduced state on the low N_A qubits
// (k_gram.cu): column-major d_A x d_A complex C; `planes` holds
// gram_plane_bytes(N, N_A) bytes; *launches receives the kernels issued.
size_t gram_plane_bytes(int N, int NA);
cudaError_t launch_gram(const float2 *psi, int N, int NA, float2 *C, void *planes, int *err, int *launches,
                        cudaStream_t st);

} // namespace sre
