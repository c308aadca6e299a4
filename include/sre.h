/*
 * sre.h -- C ABI of the GB300 (sm_103a) library for the FWHT Pauli-spectrum
 * method of Xiao & Ryu, "Exponentially Accelerated Sampling of Pauli Strings
 * for Nonstabilizerness" (arXiv 2601.00761).
 *
 * For an N-qubit state psi (d = 2^N amplitudes, complex64, amplitude psi[b]
 * of basis state |b>, qubit j = bit j of b) the library evaluates the Pauli
 * expectations
 *
 *     c_{x,z} = s * i^{popcount(x&z)} * sum_b conj(psi[b^x]) (-1)^{popcount(z&b)} psi[b],
 *     s = 1 / sum_b |psi[b]|^2,
 *
 * of the Hermitian Pauli strings P_{x,z} = i^{x.z} X^x Z^z (Eqs. Pxz-def and
 * Pxz-corr), one X-mask family {c_{x,z}}_z per Walsh-Hadamard transform
 * (Algorithm 1), and reduces them to the stabilizer Renyi entropies
 * M_1, M_2, M_3 (Eq. SRE-def; M_1 its Shannon limit; base-2 logs) and the
 * stabilizer nullity (the nullity definition with a tolerance, Algorithm 1).
 *
 * Conventions shared by every entry point
 *  - Every call returns sre_status; 0 (SRE_OK) is success. A call never
 *    aborts the process. sre_last_error() returns a message for the calling
 *    thread's last failed call.
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *    library neither frees nor keeps them after the call returns. *_host
 *    pointers are host memory owned by the caller.
 *  - psi_c64_dev is d interleaved (re, im) float pairs, 8-byte aligned. psi is
 *    normalised by the library (s above); its norm must not be zero.
 *  - stream is a cudaStream_t cast to void* (NULL = the legacy default
 *    stream). Work is issued on that stream. Calls that return results in a
 *    host struct synchronise the stream before returning.
 *  - workspace: device scratch of at least sre_workspace_bytes() bytes, owned
 *    by the caller, or NULL, in which case the library uses a buffer of its
 *    own (kept per device until sre_release_workspace()).
 *  - N is limited to 1..32 (sre_mc: 2..30, sre_exact: 1..26; see each call).
 *  - Errors: SRE_EINVAL (bad argument: N out of range, NULL or misaligned
 *    pointer, bad option), SRE_ENOMEM (allocation failed), SRE_ECUDA (a CUDA
 *    call failed; message says which), SRE_EZERO (psi has zero norm),
 *    SRE_ENULLITY (the count of |c| = 1 strings is not a power of two),
 *    SRE_ETIMEOUT (a bounded device-side wait expired), SRE_ENOTSUP
 *    (valid request this build does not serve).
 */
#ifndef SRE_H
#define SRE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SRE_API __attribute__((visibility("default")))
#else
#define SRE_API
#endif

typedef int sre_status;

#define SRE_OK 0
#define SRE_EINVAL 1
#define SRE_ENOMEM 2
#define SRE_ECUDA 3
#define SRE_EZERO 4
#define SRE_ENULLITY 5
#define SRE_ETIMEOUT 6
#define SRE_ENOTSUP 7

/* Arithmetic of the family transforms (sre_opts.precision). */
#define SRE_FP32_SIMT 0 /* FP32 butterflies on the CUDA cores */
#define SRE_BF16X2_TC 1 /* H_16 Kronecker factors on the tensor cores, data split hi+lo in BF16 */
#define SRE_BF16X3_TC 2 /* as above with a three-way BF16 split */

/* Distribution of the sampled X-masks (sre_mc mode). */
#define SRE_MC_UNIFORM 0  /* x = 0 always plus uniform x != 0: SM Sec. I estimator */
#define SRE_MC_MARGINAL 1 /* x ~ p(x) = sum_z c_{x,z}^2/d, then z ~ c_{x,z}^2/(d p(x)) */

/* Gate opcodes of sre_gate.op. */
#define SRE_GATE_H 0    /* (1/sqrt2)[[1,1],[1,-1]] on q0 */
#define SRE_GATE_S 1    /* diag(1, i) on q0 */
#define SRE_GATE_SDG 2  /* diag(1, -i) on q0 */
#define SRE_GATE_CNOT 3 /* control q0, target q1 */
#define SRE_GATE_T 4    /* diag(1, e^{i pi/4}) on q0 */
#define SRE_GATE_TDG 5  /* diag(1, e^{-i pi/4}) on q0 */

typedef struct {
    int precision;      /* SRE_FP32_SIMT (default), SRE_BF16X2_TC, SRE_BF16X3_TC */
    double eps_null;    /* nullity tolerance on | |c| - 1 |; <= 0 means 1e-6; >= 0.5 or NaN:
                           SRE_EINVAL */
    int radix_log2;     /* bits of the last (contiguous) transform pass; 0 = planned/tuned */
    int tile_log2;      /* bits per strided pass; 0 = planned/tuned */
    int x_batch;        /* X-mask families in flight per launch; 0 = planned/tuned */
    int batch_queue;    /* sre_exact_batched, FP32 only: 0 (default) = one persistent launch over the
                           single-pass states (N <= 14), chunked launches for the others; 1 = every
                           family of every state (N <= 20) in one persistent launch through a
                           dependency queue with bounded waits; other values: SRE_EINVAL */
} sre_opts;

typedef struct {
    double M[3];        /* M_1, M_2, M_3 (bits) */
    double S[3];        /* exact: H(pi) in bits, sum c^4/d^2, sum c^6/d^3;
                           MC: the estimates of -E_pi[log2 c^2], E_pi[c^2], E_pi[c^4] */
    double err_M[3];    /* exact: bound on |dM| from FP32 rounding; MC: standard error */
    double M_rb[3];     /* MC: per-family (conditional-expectation) estimator; exact: = M */
    double err_rb[3];   /* its standard error (exact: = err_M) */
    double parseval;    /* exact: sum_P c_P^2 / d (1 up to rounding, the normalisation
                           of the SRE section); MC: -1 (not computed) */
    long long stab_count; /* #{P : | |c_P| - 1 | < eps_null} (exact / nullity calls), else -1 */
    int nullity;        /* N - log2(stab_count), or -1 when not computed */
    int n_passes;       /* global transform passes per family in the plan used */
    long long n_flagged;  /* families re-evaluated in FP64 for the nullity */
    long long n_families; /* families transformed */
    long long n_samples;  /* (x, z) pairs drawn (MC marginal), else 0 */
    long long n_boundary; /* reserved (0) */
    double r2;          /* fluctuation ratio Std_{x != 0}(m_x) / E_x[m_x] of the per-family sums
                           m_x = sum_z c_{x,z}^4 that govern the uniform-x Monte Carlo estimator
                           (Supplemental Material, Clifford preconditioning): exact sweeps over all x;
                           sre_mc UNIFORM, the estimate from its sampled families; NaN otherwise */
} sre_result;

typedef struct {
    unsigned char op; /* SRE_GATE_* */
    unsigned char q0; /* qubit (control for CNOT) */
    unsigned char q1; /* CNOT target; ignored otherwise */
} sre_gate;

/* Plan of the family transform for N qubits (host only, no GPU needed). */
typedef struct {
    int N;
    int n_bits;          /* N - 1: bits of the packed complex transform */
    int n_passes;        /* 1 (whole family in one CTA) or 2..4 global passes */
    int pass_lo[4];      /* lowest bit of each pass; pass 0 reads psi, the last reduces */
    int pass_bits[4];    /* bits transformed by each pass */
    int x_batch;         /* families per launch */
    int range_log2;      /* log2 of the z-range size used by the two-level z sampler */
    size_t workspace_exact; /* bytes sre_exact needs */
} sre_plan;

/* Library version string and the last error of the calling thread. */
SRE_API const char *sre_version(void);
SRE_API const char *sre_last_error(void);

/* Fill *opts with the defaults (FP32 SIMT, eps_null 1e-6, planned tiles). */
SRE_API void sre_default_opts(sre_opts *opts);

/* Plan of the transform passes (host only). opts may be NULL. */
SRE_API sre_status sre_make_plan(int N, const sre_opts *opts, sre_plan *plan);

/* Device scratch that sre_exact (mode -1) or sre_mc (mode SRE_MC_*) needs
 * for these sizes; *bytes receives it. Host only. */
SRE_API sre_status sre_workspace_bytes(int N, int mode, long long n_x, int z_per_x,
                               const sre_opts *opts, size_t *bytes);

/* Free the library-owned workspace of the current device. */
SRE_API sre_status sre_release_workspace(void);

/* s^-1 = sum_b |psi[b]|^2 in FP64 (the normalisation of the SRE section,
 * Tr rho^2 = 1). *norm2_host receives it. */
SRE_API sre_status sre_norm2(const void *psi_c64_dev, int N, double *norm2_host, void *stream);

/* Exact enumeration of all 4^N strings, Algorithm 1: M_1..M_3 and the
 * nullity in one sweep over the 2^N X-mask families (each family one
 * Walsh-Hadamard transform of f_x, Eq. Pxz-corr). Families whose FP32
 * spectrum has |c| > 1 - eps_null - 1e-4 (n_flagged of them) are recounted
 * with every | |c| - 1 | < eps_null decision taken in FP64 (the listed
 * candidates of each such family, by direct or coset sums, or its FP64
 * transform). N in 1..26. out: host. */
SRE_API sre_status sre_exact(const void *psi_c64_dev, int N, const sre_opts *opts,
                     void *workspace, size_t workspace_bytes, void *stream,
                     sre_result *out);

/* Exact M_1..M_3 and nullity of `count` states of possibly different N in
 * one call (Algorithm 1 per state; psi_ptrs_host[i] a device pointer,
 * Ns_host[i] in 1..20). States are grouped by N. In the FP32 sweep every
 * family of every state with N <= 14 (one shared-memory tile per family) is
 * one item of a single persistent launch; each launch for N >= 15 covers the
 * (state, family) items of a chunk of same-N states. The launch sequence of
 * the whole batch is captured once into a CUDA graph (cached for the same
 * batch shape and plans) and replayed; the FP64 nullity recount of candidate
 * families follows, as in sre_exact. Plans come from sre_autotune's table when opts leaves the tiling
 * at 0. out: host array of `count` results (a state whose stabilizer count is
 * not a power of two gets nullity -1). workspace must be NULL (library
 * workspace). Returns SRE_EZERO if a state has zero norm. */
SRE_API sre_status sre_exact_batched(const void *const *psi_ptrs_host, const int *Ns_host, int count,
                             const sre_opts *opts, void *workspace, size_t workspace_bytes,
                             void *stream, sre_result *out);

/* Autotuner: times every admissible tiling (radix_log2, tile_log2, x_batch)
 * of the family transform for N on the caller's state psi and keeps the
 * fastest in a process-wide table that sre_exact, sre_exact_batched, sre_mc
 * and the plan/workspace queries use whenever opts leaves those three fields
 * at 0 (so query workspace sizes after tuning). If the environment variable
 * SRE_TUNE_FILE names a file, the table is read from and written to it.
 * *best receives the choice (the defaults when N needs a single pass). N in
 * 2..26. */
SRE_API sre_status sre_autotune(const void *psi_c64_dev, int N, void *stream, sre_opts *best);

/* Drops the autotuner's choice for N (N = 0: for every N), so that plans go
 * back to the planned defaults; rewrites SRE_TUNE_FILE when it is set. N in
 * 0..32, else SRE_EINVAL. Host only. */
SRE_API sre_status sre_autotune_clear(int N);

/* Monte Carlo over X-mask families (N in 2..30).
 * mode SRE_MC_UNIFORM: the SM Sec. I estimator -- x = 0 always and n_x - 1
 *   draws of x uniform on {1..d-1}; S_hat = m_0 + (d-1)/(n_x-1) sum m_x;
 *   err_M from Eq. stdM. z_per_x is ignored.
 * mode SRE_MC_MARGINAL: family 0 is x = 0, evaluated exactly (its own
 *   stratum, as the SM Sec. I estimator treats it); families 1..n_x-1 draw
 *   x ~ p(x | x != 0) (inverse CDF of the exact marginal over x >= 1 in
 *   natural order); every family then draws z_per_x z ~ c_{x,z}^2/(d p(x))
 *   (inverse CDF in natural z order). For g in {-log2 c^2, c^2, c^4},
 *   E_pi[g] = p(0) G_0 + (1 - p(0)) mean_i Y_i with Y_i the mean of g over
 *   family i's z draws (M, err_M) or its exact conditional mean (M_rb,
 *   err_rb); M_1 = E_pi[-log2 c^2], M_a = log2(E_pi[c^{2a-2}])/(1-a).
 * Random numbers: word 0 of Philox4x64-10 with key (seed, 0) and counter
 * (counter0 + i, lane, 0, 0); lane 0 gives family i's x, lane 1+k its k-th z;
 * u = (word >> 11) 2^-53.
 * xs_dev (n_x uint64), zs_dev (n_x*z_per_x uint64) and c_dev (n_x*z_per_x
 * float, the sampled c_{x,z}) are optional device outputs (NULL to skip).
 * out: host. */
SRE_API sre_status sre_mc(const void *psi_c64_dev, int N, int mode, long long n_x, int z_per_x,
                  unsigned long long seed, unsigned long long counter0, const sre_opts *opts,
                  void *workspace, size_t workspace_bytes, void *stream, sre_result *out,
                  unsigned long long *xs_dev, unsigned long long *zs_dev, float *c_dev);

/* The exact X-mask marginal p(x) = sum_z c_{x,z}^2 / d = (q*q)(x), the XOR
 * autocorrelation of q = s|psi|^2, computed as WHT(WHT(q)^2)/d in FP64
 * (WHT(q) is the x = 0 family, Eq. Z-FWHT). p_dev: d doubles. N in 1..30.
 * workspace: 8*d bytes or NULL. */
SRE_API sre_status pauli_x_marginal(const void *psi_c64_dev, int N, double *p_dev,
                            void *workspace, size_t workspace_bytes, void *stream);

/* Stabilizer nullity nu = N - log2 #{P : | |c_P| - 1 | < eps} (the nullity
 * definition, Algorithm 1); eps <= 0 means 1e-6, eps >= 0.5 or NaN is
 * SRE_EINVAL. N in 1..26. The FP32 sweep flags every family holding a
 * |c| > 1 - eps - 1e-4; the flagged families are recounted with every
 * | |c| - 1 | < eps decision taken in FP64. */
SRE_API sre_status stabilizer_nullity(const void *psi_c64_dev, int N, double eps, int *nullity_host,
                              long long *stab_count_host, void *stream);

/* Apply a gate list in order, in place, to psi (Clifford preconditioning and
 * T doping): H, S, S^dag, T, T^dag on q0; CNOT q0 -> q1. gates_host: n_gates
 * packed 3-byte rows. N in 1..32. Runs of gates are fused into passes over
 * psi. Returns SRE_EINVAL (and leaves psi untouched) on a bad row. */
SRE_API sre_status apply_clifford_tdoped_circuit(void *psi_c64_dev, int N, const sre_gate *gates_host,
                                         long long n_gates, void *stream);

/* Stabilizer Renyi entropy of a reduced state (Supplemental Material,
 * "Stabilizer Renyi entropy of mixed states", Eq. Msre-mixed). */
typedef struct {
    double M[3];        /* M_alpha(rho_A), alpha = 1, 2, 3, as printed (S_2 subtracted for every
                           alpha); M_1 only for a pure rho_A (Shannon limit -W[3]/d_A), else NaN */
    double S2;          /* second Renyi entropy of rho_A, -log2(W[0] / d_A) */
    double W[4];        /* over the 4^{N_A} Pauli strings supported on A: sum c^2, c^4, c^6, c^2 log2 c^2 */
    double err_M[3];    /* a-priori bound on |dM| from FP32 rounding */
    int N_A;
} sre_mixed_result;

/* Workspace bytes of sre_mixed (dominated by the d_A x d_A Gram matrix, 8 d_A^2 bytes). */
SRE_API sre_status sre_mixed_workspace_bytes(int N, int N_A, size_t *bytes);

/* SRE of rho_A, the reduced state of the first N_A qubits (the low N_A bits of
 * the basis index, b = a + 2^{N_A} e) of psi: c_P = Tr(rho_A P) for the
 * 4^{N_A} Pauli strings on A. The family x_A needs h(a) = sum_e
 * conj(psi(a ^ x_A, e)) psi(a, e), an entry of the Gram matrix C = Psi Psi^H
 * of psi viewed as a d_A x d_B matrix (one cuBLAS GEMM, FP32 emulated on the
 * BF16 tensor cores with each input split into three BF16 parts), then
 * one N_A-bit transform per x_A with the moments fused (O(2^{N+N_A}) overall).
 * N in 1..30, N_A in 1..min(N, 15). workspace: >= sre_mixed_workspace_bytes,
 * 256-byte aligned, or NULL (library-owned). out: host. Synchronises the stream. */
SRE_API sre_status sre_mixed(const void *psi_c64_dev, int N, int N_A, void *workspace, size_t workspace_bytes,
                             void *stream, sre_mixed_result *out);

/* Apply general two-qubit gates in order, in place, to psi: the random
 * brick-wall circuits of the Supplemental Material (Haar-random two-qubit
 * gates; uniformly random two-qubit Cliffords as the preconditioner C of the
 * main text). Gate k is the 4x4 complex matrix
 *   U_k[out][in] = (mats_host[32k + 2(4 out + in)], mats_host[32k + 2(4 out + in) + 1])
 * (row-major, interleaved re, im, FP32) on the ordered qubit pair
 * (pairs_host[2k], pairs_host[2k+1]) = (q0, q1), local index l = bit(q0) +
 * 2 bit(q1). Both arrays are host memory, read during the call. Runs of gates
 * inside 13 qubits are fused into one pass over psi in shared memory (gates on
 * disjoint qubits are regrouped across layers, dependencies kept). N in
 * 2..32; q0 != q1, both < N, else SRE_EINVAL with psi untouched. The matrices
 * are applied as given (unitarity is the caller's). Synchronises the stream. */
SRE_API sre_status apply_two_qubit_gates(void *psi_c64_dev, int N, const float *mats_host, const int *pairs_host,
                                         long long n_gates, void *stream);

/* One X-mask family (Eq. Pxz-corr for one x): c_dev[z] = c_{x,z} for all z,
 * d floats, by the same transform kernels as sre_exact (precision from
 * opts, NULL = FP32). N in 1..30. */
SRE_API sre_status sre_family_spectrum(const void *psi_c64_dev, int N, unsigned long long x,
                               const sre_opts *opts, float *c_dev, void *stream);

/* The same family in FP64 arithmetic (the arithmetic of the nullity
 * recheck): c_dev receives d doubles. N in 1..28. */
SRE_API sre_status sre_family_spectrum_f64(const void *psi_c64_dev, int N, unsigned long long x,
                                   double *c_dev, void *stream);

/* Philox4x64-10 blocks from the device generator that sre_mc draws with
 * (Salmon et al., SC'11): for i < n, ctr_key_dev[6i..6i+3] is the counter
 * and [6i+4..6i+5] the key; out_dev[4i..4i+3] receives the block. Lets a
 * caller check the generator against an independent implementation. */
SRE_API sre_status sre_philox_blocks(const unsigned long long *ctr_key_dev, unsigned long long *out_dev,
                             int n, void *stream);

/* Self-test of the fifth-generation tensor-core path (no counterpart in the
 * paper; it checks the conventions the tensor-core kernels rely on):
 * D = A B^T in FP32 from BF16 operands, A: M x K and B: N x K row-major
 * (K contiguous) device arrays of BF16 bit patterns, 16-byte aligned;
 * D: M x N row-major FP32. M and N multiples of 128, K of 64. swizzle: 128,
 * 64 or 32, the bytes per operand row of the shared-memory tiles (K blocks of
 * 64, 32 or 16). err_dev: a caller-owned device int the call clears and the
 * kernel sets when a bounded wait runs out (then SRE_ETIMEOUT). Synchronises
 * the stream. */
SRE_API sre_status sre_tc_gemm_selftest(const void *A_bf16_dev, const void *B_bf16_dev, float *D_dev, int M,
                                        int N, int K, int swizzle, int *err_dev, void *stream);

/* Number of CUDA kernels this library has launched since it was loaded
 * (every entry point counts its launches). Host only. */
SRE_API unsigned long long sre_kernel_launches(void);

/* Number of device allocations (cudaMalloc) this library has made since it
 * was loaded: its own per-device workspace and gate buffers, each time one is
 * created or grown. Calls given a caller workspace, and sre_exact_noalloc,
 * leave it unchanged. Host only. */
SRE_API unsigned long long sre_device_allocations(void);

/* Self-test of the bounded device waits (no counterpart in the paper). The
 * bulk-copy z sampler of sre_mc waits on mbarriers for its copies; every
 * such wait gives up after about 2^31 SM cycles (about a second), records
 * SRE_ERR_TIMEOUT in a device error word and lets the call return
 * SRE_ETIMEOUT with the context intact. This call runs one warp whose
 * mbarrier expects more bytes than the one copy issued to it, so its wait
 * can only end by the bound: it returns SRE_ETIMEOUT when the bound works
 * (about a second), SRE_OK if the wait completed (a broken barrier), or
 * SRE_ECUDA. Synchronises the stream. */
SRE_API sre_status sre_selftest_bounded_wait(void *stream);

/* Self-test of the bounded dependency waits of the persistent batched sweep
 * (no counterpart in the paper). With sre_opts.batch_queue = 1,
 * sre_exact_batched runs every family of every state as one queue of work
 * items in one launch; an item that needs earlier items (the row pass of a
 * family batch after its strided pass, a ring slot after its previous batch)
 * waits on a device counter for at most about a second of the global timer,
 * then raises SRE_ERR_TIMEOUT and an abort flag that ends the launch. This
 * test launches one row item whose strided items never run, so its wait can
 * only end by the bound: it returns SRE_ETIMEOUT (about a second) and leaves
 * the context usable. Synchronises the stream. */
SRE_API sre_status sre_selftest_queue_wait(void *stream);

/* Pass timing inside sre_mc: enable = 1 clears the counters and starts
 * recording CUDA events around every full-batch family-transform pass launch
 * of subsequent sre_mc calls; enable = 0 stops. Either call first copies the
 * current counters out: ms_sum_host[p] (total ms of pass p's launches),
 * launches_host[p] (their count) and bytes_host[p] (algorithmic bytes per
 * launch, as for sre_profile_passes); each array has 4 entries, any may be
 * NULL. Host only. */
SRE_API sre_status sre_pass_timing(int enable, double *ms_sum_host, long long *launches_host,
                                   double *bytes_host);

/* Profiling aid: runs n_x families (x drawn uniformly, seed fixed) through
 * exactly the launch sequence of the family transform that sre_mc issues
 * (norm, the planned passes, fused moments epilogue), with CUDA events on
 * `stream` around every pass launch. ms_host[p] receives the mean duration of
 * pass p's launches, bytes_host[p] the algorithmic bytes one launch of pass p
 * moves (first pass: 8 B per psi amplitude read; each boundary between
 * passes: the packed intermediate, 4 B per Pauli string written and 4 B
 * read); *n_passes the pass count (<= 4); *fam_per_launch the families one
 * launch processes. Uses the library workspace. N in 2..30. */
SRE_API sre_status sre_profile_passes(const void *psi_c64_dev, int N, long long n_x, const sre_opts *opts,
                                      void *stream, double *ms_host, double *bytes_host, int *n_passes,
                                      long long *fam_per_launch);

/* sre_exact without any device allocation. The paper has no counterpart:
 * this is a deployment variant for callers that cannot allocate device memory
 * at call time -- a process whose device memory is held entirely by another
 * allocator (a framework's caching pool) or that runs under a fixed memory
 * budget, where a cudaMalloc could fail, and latency-sensitive callers that
 * cannot afford the device-wide synchronisation cudaMalloc/cudaFree can imply.
 * It runs the same launch sequence as sre_exact on a scratch array that the
 * library reserves statically (SRE_NOALLOC_SCRATCH_BYTES on every GPU that
 * loads the library, held until the process exits); psi, the stream and the
 * host result are the caller's as for sre_exact.
 *  - N is limited to 1..SRE_NOALLOC_MAX_N; larger N returns SRE_EINVAL with a
 *    message naming the limit, before any device work.
 *  - The first call on a device looks up the scratch's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call uses the same scratch and leaves its contents behind; the
 *    call clears what must start at zero. Calls whose device work overlaps
 *    (different streams, threads or processes sharing the context) race on
 *    the scratch: serialise them. */
#define SRE_NOALLOC_SCRATCH_BYTES (2u << 20)
#define SRE_NOALLOC_MAX_N 13
SRE_API sre_status sre_exact_noalloc(const void *psi_c64_dev, int N, const sre_opts *opts, void *stream,
                                     sre_result *out);

#ifdef __cplusplus
}
#endif

#endif /* SRE_H */
