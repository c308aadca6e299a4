// sre_api.cu -- the C ABI (include/sre.h): argument checks, transform plans,
// workspace layout and the launch sequences of each entry point.
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "sre.h"
#include "k_misc.cuh"
#include "k_pass_dispatch.cuh"
#include "k_batch.cuh"

using namespace sre;

namespace {

thread_local std::string g_err;

sre_status fail(sre_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return fail(SRE_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define CS(call)                          \
    do {                                  \
        sre_status s_ = (call);           \
        if (s_ != SRE_OK) return s_;      \
    } while (0)

constexpr size_t BATCH_BYTES = 8ULL << 30;   // intermediate budget per launch sequence
// FP32 states whose families exceed a quarter of that budget (N >= 29) still
// take BATCH_MIN_LARGE families per launch, within BATCH_BYTES_LARGE: the
// families of a launch share psi's reads (N = 30 MC: 5.81 ms per family at 2
// per launch, 4.94 at 8, 4.87 at 16)
constexpr long long BATCH_MIN_LARGE = 8;
constexpr size_t BATCH_BYTES_LARGE = 32ULL << 30;

// kernels issued by this library since load (all entry points)
std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
// device allocations this library made since load (cudaMalloc of its own
// workspace and gate buffers)
std::atomic<unsigned long long> g_allocs{0};
constexpr int EXACT_PARTS = 1024;

// --------------------------------------------------------------- plans
struct Plan {
    int N = 0, n = 0, prec = 32;
    int npass = 1, nstrided = 0;
    int K[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0}, ms[4] = {0, 0, 0, 0};
    int M_last = 0;
    int RL = 0;                  // log2 of the z-range size of the two-level sampler
    long long tiles_last = 1;
    long long B = 1;
    size_t slot_bytes = 0;
};

int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// z-ranges of 2^ZR_FINE z (weights written by the last pass, draws resolved by
// the folding sampler) for multi-pass plans whose last tiles are larger
bool fine_ranges(const Plan &P) { return P.npass > 1 && P.M_last > ZR_FINE; }

// ------------------------------------------------------------ autotuner table
// Best (radix_log2, tile_log2, x_batch) per N found by sre_autotune; used when
// the caller leaves all three options at 0. Optionally persisted in the file
// named by SRE_TUNE_FILE (lines "N radix tile x_batch").
struct TuneEntry { int radix = 0, tile = 0, xbatch = 0; bool valid = false; };
std::mutex g_tune_mu;
TuneEntry g_tune[33];
bool g_tune_loaded = false;

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *fn = getenv("SRE_TUNE_FILE");
    if (!fn) return;
    FILE *f = fopen(fn, "r");
    if (!f) return;
    int N, r, t, b;
    while (fscanf(f, "%d %d %d %d", &N, &r, &t, &b) == 4)
        if (N >= 1 && N <= 32) { g_tune[N].radix = r; g_tune[N].tile = t; g_tune[N].xbatch = b; g_tune[N].valid = true; }
    fclose(f);
}

void tune_save_locked() {
    const char *fn = getenv("SRE_TUNE_FILE");
    if (!fn) return;
    FILE *f = fopen(fn, "w");
    if (!f) return;
    for (int N = 1; N <= 32; ++N)
        if (g_tune[N].valid) fprintf(f, "%d %d %d %d\n", N, g_tune[N].radix, g_tune[N].tile, g_tune[N].xbatch);
    fclose(f);
}

sre_status plan_for(int N, const sre_opts *o, int prec, Plan &P);

sre_status plan_for_tuned(int N, const sre_opts *o, int prec, Plan &P) {
    sre_opts t;
    sre_default_opts(&t);
    if (o) t = *o;
    if (prec == 32 && t.radix_log2 == 0 && t.tile_log2 == 0 && t.x_batch == 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        if (N >= 1 && N <= 32 && g_tune[N].valid) {
            t.radix_log2 = g_tune[N].radix;
            t.tile_log2 = g_tune[N].tile;
            t.x_batch = g_tune[N].xbatch;
        }
    }
    return plan_for(N, &t, prec, P);
}

sre_status plan_for(int N, const sre_opts *o, int prec, Plan &P) {
    P = Plan();
    P.N = N;
    P.n = N - 1;
    P.prec = prec;
    const int single_max = prec == 32 ? F32_SINGLE_MMAX : F64_SINGLE_MMAX;
    if (P.n <= single_max) {
        P.npass = 1;
        P.M_last = P.n;
        P.RL = P.n;
        P.tiles_last = 1;
        P.slot_bytes = 0;
        P.B = 1LL << 20;
        if (prec == 32 && o && o->x_batch > 0) P.B = o->x_batch;
        return SRE_OK;
    }
    int nlo, kmax;
    if (prec == 32) {
        nlo = (o && o->radix_log2 > 0) ? clampi(o->radix_log2, F32_ROW_MMIN, F32_ROW_MMAX) : 13;
        kmax = (o && o->tile_log2 > 0) ? clampi(o->tile_log2, 1, F32_STRIDED_KMAX) : F32_STRIDED_KMAX;
    } else {
        nlo = F64_ROW_M;
        kmax = F64_STRIDED_KMAX;
    }
    auto ms_of = [&](int K) { return prec == 32 ? f32_strided_ms(K) : F64_STRIDED_M; };
    // A strided tile is 2^K rows x 2^(ms-K) columns and its columns must fit
    // below the pass's row stride 2^lo: ms - K <= lo. Only the bottom strided
    // pass (lo = nlo) can violate it: K_bottom >= 13 - nlo.
    const int rest = P.n - nlo;
    const int kmin_bottom = 13 - nlo > 1 ? 13 - nlo : 1;
    if (kmax < kmin_bottom) kmax = kmin_bottom;
    int ns = (rest + kmax - 1) / kmax;
    if (ns > 3) return fail(SRE_ENOTSUP, "N=%d needs %d strided passes", N, ns);
    // balanced, extra bits to the lower passes
    for (int i = 0; i < ns; ++i) P.K[i] = rest / ns + (i >= ns - rest % ns ? 1 : 0);
    if (P.K[ns - 1] < kmin_bottom) {
        if (rest < kmin_bottom) return fail(SRE_EINVAL, "N=%d: radix %d leaves %d strided bits", N, nlo, rest);
        P.K[ns - 1] = kmin_bottom;
        const int rem = rest - kmin_bottom;
        const int no = ns - 1 > 0 ? ns - 1 : (rem > 0 ? 1 : 0);
        if (no + 1 > 3) return fail(SRE_ENOTSUP, "N=%d needs %d strided passes", N, no + 1);
        for (int i = 0; i < no; ++i) P.K[i] = rem / no + (i >= no - rem % no ? 1 : 0);
        P.K[no] = kmin_bottom;
        ns = no + 1;
    }
    P.nstrided = ns;
    P.npass = ns + 1;
    int top = P.n;
    for (int i = 0; i < ns; ++i) {
        P.lo[i] = top - P.K[i];
        P.ms[i] = ms_of(P.K[i]);
        top = P.lo[i];
        if (P.ms[i] - P.K[i] > P.lo[i]) return fail(SRE_EINVAL, "internal plan error (N=%d pass %d)", N, i);
    }
    P.M_last = nlo;
    P.tiles_last = 1LL << (P.n - nlo);
    P.slot_bytes = (size_t)(prec == 32 ? 8 : 16) << P.n;
    long long B = (long long)(BATCH_BYTES / P.slot_bytes);
    if (prec == 32 && B < BATCH_MIN_LARGE)
        B = std::min(BATCH_MIN_LARGE, (long long)(BATCH_BYTES_LARGE / P.slot_bytes));
    if (B < 1) B = 1;
    if (B > 4096) B = 4096;
    if (prec == 32 && o && o->x_batch > 0) B = o->x_batch;
    P.B = B;
    P.RL = fine_ranges(P) ? ZR_FINE : P.M_last;
    return SRE_OK;
}

// -------------------------------------------------------------- arena
struct Arena {
    char *base;
    size_t off = 0;
    explicit Arena(void *b) : base((char *)b) {}
    template <class T> T *take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += n * sizeof(T) + 256;
        return p;
    }
};

// Nullity recount of flagged families (FP64 decisions): an FP32 pass lists
// each family's candidate z' (NULL_CHUNK families at a time); families with
// few candidates are recounted by direct FP64 sums at them, the rest by the
// FP64 transform.
constexpr long long NULL_CHUNK = 1LL << 11;

struct NullWS {
    unsigned *cand_cnt, *cand_z;      // per chunk: counts, lists [slot][NULL_CAND_MAX]
    unsigned long long *counts;       // per flagged family (direct recount; 0 for the overflow)
    unsigned long long *ovf, *ovf_n;  // overflow families (capacity: the flagged families)
    unsigned long long *counts2;      // per overflow family (FP64 transform)
    void *inter, *inter64;
};

void layout_null(Arena &A, long long fam_cap, NullWS &w) {
    const long long ch = std::min(fam_cap, NULL_CHUNK);
    w.cand_cnt = A.take<unsigned>((size_t)ch);
    w.cand_z = A.take<unsigned>((size_t)ch * NULL_CAND_MAX);
    w.ovf = A.take<unsigned long long>((size_t)fam_cap);
    w.ovf_n = A.take<unsigned long long>(1);
    w.counts2 = A.take<unsigned long long>((size_t)fam_cap);
}

struct ExactWS {
    double *scal, *npart, *epart, *etot;
    void *inter;
    TilePartial *tiles;
    FamMoments *fm;
    unsigned long long *flags, *nflag, *counts, *cnt_sum;
    void *inter64;
    NullWS nw;
};

void layout_exact(Arena &A, const Plan &P, const Plan &P64, ExactWS &w) {
    const unsigned long long d = 1ULL << P.N;
    w.scal = A.take<double>(SCAL_N);
    w.npart = A.take<double>(NORM_BLOCKS);
    w.epart = A.take<double>(6 * EXACT_PARTS);
    w.etot = A.take<double>(8);
    w.inter = P.npass > 1 ? (void *)A.take<char>(P.slot_bytes * (size_t)P.B) : nullptr;
    const long long nb = P.npass > 1 ? P.B : (long long)d;
    w.tiles = A.take<TilePartial>((size_t)nb * (size_t)P.tiles_last);
    w.fm = A.take<FamMoments>(d);
    w.flags = A.take<unsigned long long>(d);
    w.nflag = A.take<unsigned long long>(1);
    w.counts = A.take<unsigned long long>(d);
    w.cnt_sum = A.take<unsigned long long>(2);
    w.inter64 = P64.npass > 1 ? (void *)A.take<char>(P64.slot_bytes * (size_t)P64.B) : nullptr;
    layout_null(A, (long long)d, w.nw);
    w.nw.counts = w.counts;
    w.nw.inter = w.inter;
    w.nw.inter64 = w.inter64;
}

struct McWS {
    double *scal, *npart;
    double *p, *mwork, *bsum;
    unsigned long long *xs;
    unsigned long long *xs_ord, *perm;   // the families in processing order, and their own indices
    void *inter;
    TilePartial *tiles;
    FamMoments *fm;
    float *Wf;       // range weights (FP32, one row per family of the batch)
    DrawInfo *draws;
    unsigned long long *zs;
    float *cz;
    double *y, *out;
    int *err;        // device error word (SRE_ERR_* bits)
};

void layout_mc(Arena &A, const Plan &P, int mode, long long n_x, int zpx, McWS &w) {
    const unsigned long long d = 1ULL << P.N;
    const bool marg = mode == SRE_MC_MARGINAL;
    w.scal = A.take<double>(SCAL_N);
    w.npart = A.take<double>(NORM_BLOCKS);
    w.p = marg ? A.take<double>(d) : nullptr;
    w.mwork = marg ? A.take<double>(d) : nullptr;
    w.bsum = marg ? A.take<double>(d / SCAN_CHUNK + 1) : nullptr;
    w.xs = A.take<unsigned long long>(n_x);
    w.xs_ord = P.npass > 1 ? A.take<unsigned long long>(n_x) : nullptr;
    w.perm = P.npass > 1 ? A.take<unsigned long long>(n_x) : nullptr;
    const long long B = P.npass > 1 ? P.B : (n_x < P.B ? n_x : P.B);
    w.inter = P.npass > 1 ? (void *)A.take<char>(P.slot_bytes * (size_t)P.B) : nullptr;
    w.tiles = A.take<TilePartial>((size_t)B * (size_t)P.tiles_last);
    w.fm = A.take<FamMoments>(n_x);
    const long long nr = 1LL << (P.N - P.RL);
    w.Wf = marg ? A.take<float>((size_t)B * (size_t)nr) : nullptr;
    const size_t nd = marg ? (size_t)n_x * (size_t)zpx : 1;
    w.draws = marg ? A.take<DrawInfo>(nd) : nullptr;
    w.zs = marg ? A.take<unsigned long long>(nd) : nullptr;
    w.cz = A.take<float>(nd);
    w.y = A.take<double>(6 * (size_t)n_x);
    w.out = A.take<double>(24);
    w.err = A.take<int>(1);
}

// ------------------------------------------------ library-owned workspace
std::mutex g_ws_mu;
struct DevWS { void *p = nullptr; size_t n = 0; };
std::vector<DevWS> g_ws;
struct DevBuf { void *p = nullptr; size_t n = 0; };
std::vector<DevBuf> g_gatebuf;

sre_status own_workspace(size_t need, void **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if ((int)g_ws.size() <= dev) g_ws.resize(dev + 1);
    DevWS &w = g_ws[dev];
    if (w.n < need) {
        if (w.p) CK(cudaFree(w.p));
        w.p = nullptr;
        w.n = 0;
        cudaError_t e = cudaMalloc(&w.p, need);
        g_allocs.fetch_add(1, std::memory_order_relaxed);
        if (e != cudaSuccess) {
            w.p = nullptr;
            return fail(SRE_ENOMEM, "cudaMalloc(%zu) failed: %s", need, cudaGetErrorString(e));
        }
        w.n = need;
    }
    *out = w.p;
    return SRE_OK;
}

sre_status resolve_workspace(void *ws, size_t ws_bytes, size_t need, void **out) {
    if (ws) {
        if (ws_bytes < need) return fail(SRE_EINVAL, "workspace of %zu bytes, %zu needed", ws_bytes, need);
        if (((uintptr_t)ws) & 255) return fail(SRE_EINVAL, "workspace must be 256-byte aligned");
        *out = ws;
        return SRE_OK;
    }
    return own_workspace(need, out);
}

// ------------------------------------------------------------ checks
sre_status check_psi(const void *psi, int N, int nmin, int nmax) {
    if (N < nmin || N > nmax) return fail(SRE_EINVAL, "N=%d outside %d..%d", N, nmin, nmax);
    if (!psi) return fail(SRE_EINVAL, "psi is NULL");
    if (((uintptr_t)psi) & 7) return fail(SRE_EINVAL, "psi must be 8-byte aligned");
    return SRE_OK;
}

sre_status check_opts(const sre_opts *o, sre_opts &out) {
    sre_default_opts(&out);
    if (!o) return SRE_OK;
    out = *o;
    if (out.eps_null <= 0) out.eps_null = 1e-6;
    if (!(out.eps_null < 0.5)) return fail(SRE_EINVAL, "eps_null must lie in (0, 0.5)");
    if (out.precision != SRE_FP32_SIMT && out.precision != SRE_BF16X2_TC && out.precision != SRE_BF16X3_TC)
        return fail(SRE_EINVAL, "unknown precision %d", out.precision);
    if (out.x_batch < 0 || out.radix_log2 < 0 || out.tile_log2 < 0)
        return fail(SRE_EINVAL, "negative tiling option");
    if (out.batch_queue != 0 && out.batch_queue != 1) return fail(SRE_EINVAL, "batch_queue must be 0 or 1");
    return SRE_OK;
}

// FP32 candidate threshold for the nullity tolerance eps: a c with
// | |c| - 1 | < eps has |c| > 1 - eps, and the FP32 (or split-BF16) |c| is
// within 1e-5 of the FP64 one, so 1e-4 below 1 - eps misses none of them.
float cand_threshold(double eps) { return (float)(1.0 - eps - 1e-4); }

// Listed z' per family up to which direct FP64 sums (4 + 2k operations per
// packed point) undercut the FP64 transform (about 2N + 8).
int null_kdirect(int N) { return std::min(NULL_CAND_MAX, N + 2); }

PassArgs base_args(const Plan &P, const void *psi, const double *scal) {
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.psi = reinterpret_cast<const float2 *>(psi);
    a.N = P.N;
    a.n = P.n;
    a.slot_elems = 1LL << P.n;
    a.range_log2 = P.RL;
    a.s_ptr = scal + SCAL_S;
    a.cand_thr = 1.0f - 1e-4f;
    a.want_cand = 1;
    a.precision = 0;
    return a;
}

// precision code of the FP32 family transforms for the kernels
int prec_code(const sre_opts &o) {
    return o.precision == SRE_BF16X3_TC ? 3 : (o.precision == SRE_BF16X2_TC ? 2 : 0);
}


// Optional CUDA-event timing of every pass launch.
struct PassTimer {
    std::vector<cudaEvent_t> ev;   // pairs (start, stop) per launch
    std::vector<int> pass;         // pass index of each pair
};

sre_status timer_mark(PassTimer *T, int pass, cudaStream_t st, bool start) {
    if (!T) return SRE_OK;
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    CK(cudaEventRecord(e, st));
    T->ev.push_back(e);
    if (start) T->pass.push_back(pass);
    return SRE_OK;
}

// Library-wide pass timing (sre_pass_timing): when on, run_transform of the
// FP32 family transforms records events around each pass launch and the
// entry point folds them into per-pass sums after its stream synchronisation.
std::mutex g_timing_mu;
bool g_timing_on = false;
double g_timing_ms[4] = {0, 0, 0, 0};
long long g_timing_n[4] = {0, 0, 0, 0};
double g_timing_bytes[4] = {0, 0, 0, 0};

sre_status timer_fold(PassTimer &T) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    for (size_t i = 0; i < T.pass.size(); ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, T.ev[2 * i], T.ev[2 * i + 1]));
        g_timing_ms[T.pass[i]] += ms;
        g_timing_n[T.pass[i]] += 1;
    }
    for (cudaEvent_t e : T.ev) cudaEventDestroy(e);
    T.ev.clear();
    T.pass.clear();
    return SRE_OK;
}

void timing_bytes(const Plan &P, long long fam_per_launch) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    const double d = std::ldexp(1.0, P.N);
    for (int p = 0; p < P.npass; ++p) {
        double b = 0.0;
        if (p == 0) b += 8.0 * d;
        if (p > 0) b += 4.0 * d;
        if (p < P.npass - 1) b += 4.0 * d;
        g_timing_bytes[p] = b * (double)fam_per_launch;
    }
}

// One transform of every family in a.fam_base .. + a.n_fam (one launch
// sequence): strided passes top-down, then the last pass with dst_last.
sre_status run_transform(const Plan &P, PassArgs a, int src0, int dst_last, void *inter, cudaStream_t st,
                         PassTimer *T = nullptr) {
    cudaError_t e;
    if (P.npass == 1) {
        a.lo_g = 0;
        CS(timer_mark(T, 0, st, true));
        e = P.prec == 32 ? launch_f32_single(P.n, src0, dst_last, a, st) : launch_f64_single(P.n, src0, dst_last, a, st);
        if (e != cudaSuccess) return fail(SRE_ECUDA, "single-pass launch (N=%d): %s", P.N, cudaGetErrorString(e));
        count_launches(1);
        CS(timer_mark(T, 0, st, false));
        return SRE_OK;
    }
    for (int i = 0; i < P.nstrided; ++i) {
        PassArgs b = a;
        b.lo_g = P.lo[i];
        b.src = inter;
        b.dst = inter;
        const int s = i == 0 ? src0 : SRC_BUF;
        CS(timer_mark(T, i, st, true));
        const int tiles = (int)(1LL << (P.n - P.ms[i]));
        e = P.prec == 32 ? launch_f32_strided(P.ms[i], P.K[i], s, DST_BUF, b, tiles, st)
                         : launch_f64_strided(P.K[i], s, DST_BUF, b, tiles, st);
        if (e != cudaSuccess)
            return fail(SRE_ECUDA, "strided pass %d (N=%d K=%d): %s", i, P.N, P.K[i], cudaGetErrorString(e));
        count_launches(1);
        CS(timer_mark(T, i, st, false));
    }
    PassArgs b = a;
    b.lo_g = 0;
    b.src = inter;
    if (dst_last == DST_SQMAP) b.dst = inter;
    CS(timer_mark(T, P.nstrided, st, true));
    e = P.prec == 32 ? launch_f32_row(P.M_last, SRC_BUF, dst_last, b, (int)P.tiles_last, st)
                     : launch_f64_row(P.M_last, SRC_BUF, dst_last, b, (int)P.tiles_last, st);
    if (e != cudaSuccess) return fail(SRE_ECUDA, "row pass (N=%d): %s", P.N, cudaGetErrorString(e));
    count_launches(1);
    CS(timer_mark(T, P.nstrided, st, false));
    return SRE_OK;
}

// x-marginal into p (FP64): WHT(|psi|^2) -> square -> WHT -> /d
sre_status run_marginal(const void *psi, int N, const double *scal, double *p, double *mwork, cudaStream_t st) {
    Plan P64;
    CS(plan_for(N, nullptr, 64, P64));
    PassArgs a = base_args(P64, psi, scal);
    a.n_fam = 1;
    a.dst = mwork;
    a.src = mwork;
    a.p_out = p;
    CS(run_transform(P64, a, SRC_PSI_Q, DST_SQMAP, mwork, st));
    CS(run_transform(P64, a, SRC_BUF, DST_P, mwork, st));
    return SRE_OK;
}

// Recount of the n flagged families xs (F, with the state in the high bits
// when a32.psi_list is set): counts[i] per family from the coset or direct
// FP64 sums (k_null.cu); the families that neither route takes land in ovf
// (*n_ovf of them) with their FP64-transform counts in counts2.
sre_status null_recount(const Plan &P, const Plan &P64, const PassArgs &a32, const PassArgs &a64,
                        const unsigned long long *xs, long long n, double eps, const NullWS &w, cudaStream_t st,
                        long long *n_ovf) {
    CK(cudaMemsetAsync(w.ovf_n, 0, sizeof(unsigned long long), st));
    PassArgs c = a32;
    c.xs = xs;
    c.precision = 0;
    c.want_cand = 0;
    c.cand_thr = cand_threshold(eps);
    c.cand_cnt = w.cand_cnt;
    c.cand_z = w.cand_z;
    c.cand_max = NULL_CAND_MAX;
    NullDirectArgs q;
    memset(&q, 0, sizeof q);
    q.psi = a32.psi;
    q.s_ptr = a32.s_ptr;
    q.psi_list = a32.psi_list;
    q.s_list = a32.s_list;
    q.N = P.N;
    q.xs = xs;
    q.cand_cnt = w.cand_cnt;
    q.cand_z = w.cand_z;
    q.cand_max = NULL_CAND_MAX;
    q.kdirect = null_kdirect(P.N);
    q.eps = eps;
    q.ovf = w.ovf;
    q.ovf_n = w.ovf_n;
    const long long chunk = P.npass > 1 ? std::min(P.B, NULL_CHUNK) : NULL_CHUNK;
    for (long long fb = 0; fb < n; fb += chunk) {
        const long long nf = std::min(chunk, n - fb);
        CK(cudaMemsetAsync(w.cand_cnt, 0, sizeof(unsigned) * (size_t)nf, st));
        PassArgs b = c;
        b.fam_base = fb;
        b.n_fam = nf;
        CS(run_transform(P, b, SRC_PSI_FAMILY, DST_CANDLIST, w.inter, st));
        q.fam_base = fb;
        q.counts = w.counts + fb;
        CK(launch_null_direct(q, nf, st));
        count_launches(1);
    }
    unsigned long long no = 0;
    CK(cudaMemcpyAsync(&no, w.ovf_n, sizeof no, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (no > 0) {
        CK(cudaMemsetAsync(w.counts2, 0, sizeof(unsigned long long) * no, st));
        PassArgs d = a64;
        d.xs = w.ovf;
        d.eps = eps;
        const long long step64 = P64.npass > 1 ? P64.B : (1LL << 20);
        for (long long fb = 0; fb < (long long)no; fb += step64) {
            PassArgs e = d;
            e.fam_base = fb;
            e.n_fam = std::min(step64, (long long)no - fb);
            e.count_out = w.counts2 + fb;
            CS(run_transform(P64, e, SRC_PSI_FAMILY, DST_NULLCOUNT, w.inter64, st));
        }
    }
    *n_ovf = (long long)no;
    return SRE_OK;
}

static_assert(offsetof(sre_result, stab_count) == 128 && offsetof(sre_result, r2) == 176 &&
                  sizeof(sre_result) == 184, "sre_result layout is part of the ABI");

// Fluctuation ratio of the per-family sums m_x = sum_z c_{x,z}^4 (SM, Clifford
// preconditioning): r_2 = Std_{x != 0}(m_x) / E_x[m_x], population moments over
// the d - 1 families x != 0 and the mean over all d (a ratio: the
// normalisation of m_x cancels). sum_all = sum_x m_x, sq_nz = sum_{x != 0} m_x^2.
double fluctuation_ratio(double sum_all, double sq_nz, double m_x0, double d) {
    if (d < 2.0) return std::nan("");
    const double mean_nz = (sum_all - m_x0) / (d - 1.0);
    double var = sq_nz / (d - 1.0) - mean_nz * mean_nz;
    if (var < 0.0) var = 0.0;
    const double mean_all = sum_all / d;
    return mean_all > 0.0 ? std::sqrt(var) / mean_all : std::nan("");
}

// T: the TOT_N totals of an exact sweep (k_misc.cuh)
// pi_P = c_P^2 / (d P) with P = sum_P c_P^2 / d the measured Parseval sum (1
// in exact arithmetic for the normalised state): normalising by it cancels
// the common scale error of the FP32 (or split-BF16) spectrum, which Eq.
// SRE-def would otherwise carry N-fold into M_1 and twofold into M_2.
void finalize_exact(const double *T, int N, sre_result *r) {
    const double d = std::ldexp(1.0, N);
    const double P = T[0] / d;
    const double H = N + std::log2(P) - T[3] / (d * P);
    r->S[0] = H;
    r->S[1] = T[1] / (d * d * P * P);
    r->S[2] = T[2] / (d * d * d * P * P * P);
    r->M[0] = H - N;
    r->M[1] = -std::log2(r->S[1]) - N;
    r->M[2] = -0.5 * std::log2(r->S[2]) - N;
    r->parseval = T[0] / d;
    // a-priori FP32 rounding estimate: relative error of c ~ (N + 2) 2^-24
    const double ec = (N + 2) * std::ldexp(1.0, -24);
    r->err_M[0] = 2.0 * ec * (N + 2);
    r->err_M[1] = 4.0 * ec / std::log(2.0);
    r->err_M[2] = 6.0 * ec / (2.0 * std::log(2.0));
    for (int a = 0; a < 3; ++a) { r->M_rb[a] = r->M[a]; r->err_rb[a] = r->err_M[a]; }
    r->r2 = fluctuation_ratio(T[1], T[5], T[6], d);
}

void init_result(sre_result *r) {
    memset(r, 0, sizeof *r);
    r->stab_count = -1;
    r->nullity = -1;
    r->r2 = std::nan("");
}

sre_status nullity_from_count(long long cnt, int N, sre_result *r) {
    r->stab_count = cnt;
    if (cnt <= 0 || (cnt & (cnt - 1)) != 0) {
        r->nullity = -1;
        return fail(SRE_ENULLITY, "stabilizer count %lld is not a power of two", cnt);
    }
    int l = 0;
    while ((1LL << l) < cnt) ++l;
    r->nullity = N - l;
    return SRE_OK;
}

// exact sweep; with_moments=false still computes them (they are free)
sre_status exact_impl(const void *psi, int N, const sre_opts &o, void *ws, size_t ws_bytes, cudaStream_t st,
                      sre_result *out) {
    Plan P, P64;
    CS(plan_for_tuned(N, &o, 32, P));
    CS(plan_for(N, nullptr, 64, P64));
    Arena dry(nullptr);
    ExactWS w;
    layout_exact(dry, P, P64, w);
    void *base = nullptr;
    CS(resolve_workspace(ws, ws_bytes, dry.off, &base));
    Arena A(base);
    layout_exact(A, P, P64, w);

    const unsigned long long d = 1ULL << N;
    CK(launch_norm2((const float2 *)psi, N, w.scal, w.npart, st));
    count_launches(2);
    PassArgs a = base_args(P, psi, w.scal);
    a.precision = prec_code(o);
    a.tile_out = w.tiles;
    a.cand_thr = cand_threshold(o.eps_null);
    const long long step = P.npass > 1 ? P.B : (long long)d;
    for (long long fb = 0; fb < (long long)d; fb += step) {
        const long long nf = (long long)d - fb < step ? (long long)d - fb : step;
        PassArgs b = a;
        b.fam_base = fb;
        b.n_fam = nf;
        CS(run_transform(P, b, SRC_PSI_FAMILY, DST_MOMENTS, w.inter, st));
        CK(launch_fam_reduce(w.tiles, nf, (int)P.tiles_last, nullptr, fb, N, P.M_last, P.M_last, w.fm, fb, nullptr,
                             0, st));
        count_launches(1);
    }
    CK(cudaMemsetAsync(w.nflag, 0, sizeof(unsigned long long), st));
    CK(launch_exact_totals(w.fm, (long long)d, w.epart, EXACT_PARTS, w.etot, w.flags, w.nflag, st));
    count_launches(2);
    double host[TOT_N + 1];
    unsigned long long nflag = 0;
    CK(cudaMemcpyAsync(host, w.etot, TOT_N * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&nflag, w.nflag, sizeof nflag, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(host + TOT_N, w.scal + SCAL_NORM2, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!(host[TOT_N] > 0.0)) return fail(SRE_EZERO, "psi has zero norm");

    // FP64 recount of the candidate families
    unsigned long long cnt = 0;
    if (nflag > 0) {
        long long no = 0;
        CS(null_recount(P, P64, base_args(P, psi, w.scal), base_args(P64, psi, w.scal), w.flags, (long long)nflag,
                        o.eps_null, w.nw, st, &no));
        CK(launch_sum_u64(w.counts, (long long)nflag, w.cnt_sum, st));
        count_launches(1);
        unsigned long long c2[2] = {0, 0};
        if (no > 0) {
            CK(launch_sum_u64(w.nw.counts2, no, w.cnt_sum + 1, st));
            count_launches(1);
        }
        CK(cudaMemcpyAsync(c2, w.cnt_sum, sizeof(unsigned long long) * (no > 0 ? 2 : 1), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        cnt = c2[0] + c2[1];
    }
    init_result(out);
    finalize_exact(host, N, out);
    out->n_flagged = (long long)nflag;
    out->n_families = (long long)d;
    out->n_passes = P.npass;
    return nullity_from_count((long long)cnt, N, out);
}


// ---------------------------------------------------------------- batched
// Exact sweeps of many states of possibly different N (sre_exact_batched).
// States are grouped by N into buckets. For each bucket one launch sequence
// covers every (state, family) item of a chunk of states: the pass kernels
// resolve the family index F = (state << N) | x into the state's psi and s.
// Per-state totals come from a fixed-order segmented reduction. The whole
// sequence of every bucket is captured once into a CUDA graph (cached per
// batch shape and workspace) and replayed; the FP64 nullity recheck of the
// candidate families follows as a second, short sequence.
constexpr long long BATCH_CHUNK_FAMILIES = 1LL << 21;

struct BucketPlan {
    int N;
    std::vector<int> idx;       // caller indices of the bucket's states
    int off;                    // first slot of the bucket in the per-state arrays
    Plan P, P64;
    int states_per_chunk;
    unsigned long long *flags;  // flagged families of the bucket (capacity: its families)
    long long flag_cap;
    bool persistent;            // swept by the persistent launch (single-pass FP32 tiles)
};

struct BatchWS {
    const float2 **psi_list;
    double *s_list, *norm_list, *npart, *totals;
    unsigned long long *state_count, *nflag, *counts;
    FamMoments *fm;
    TilePartial *tiles;
    void *inter, *inter64;
    NullWS nw;
    // the persistent launch (k_batch.cu)
    FamMoments *fm_all;                  // family sums of every state it sweeps, bucket by bucket
    BatchBucket *pbuckets;
    BatchSeg *psegs;
    unsigned long long *next;
    // with two-pass items (the dependency queue)
    unsigned *need, *done;               // per global batch: [need_str, need_row], [done_str, done_row]
    int *abort_flag, *err;
    void *ring;
    TilePartial *ring_tiles;
};

// The persistent launch's work layout, built on the host (k_batch.cuh). By
// default it holds the families of every single-pass FP32 bucket (N <= 14),
// one segment per bucket, G families per item (the tile's groups), and the
// two-pass buckets keep the chunked launch sequence (batch_main). With
// sre_opts.batch_queue it holds every bucket: the two-pass ones (N = 15 .. 20)
// as batches of strided items (a pass of N - 14 rows) and row items (13-bit
// rows with the fused moments) through an intermediate ring, in dependency
// order.
constexpr int PERSIST_SINGLE_NMAX = 14;
constexpr int PERSIST_NMAX = 20;
constexpr int PERSIST_AHEAD = 1;                      // strided batches issued ahead of a batch's row items
constexpr int PERSIST_RING = PERSIST_AHEAD + 2;       // intermediate ring slots
constexpr size_t PERSIST_SLOT_BYTES = 1ull << 30;    // intermediate bytes per ring slot (4096 families at N = 16)
constexpr int PERSIST_FPC = 8;                        // families per strided item
constexpr int PERSIST_RPI = 2;                        // families per row item

struct PersistLayout {
    bool dep = false;                                 // two-pass items queued
    std::vector<BatchBucket> buckets;                 // one per bucket of the batch (unused when not swept)
    std::vector<BatchSeg> segs;
    std::vector<size_t> fm_off;                       // first family of each bucket in fm_all
    std::vector<unsigned> need_str, need_row;         // per global batch
    long long n_items = 0;
    int batches = 0;
    size_t fm_total = 0, tiles_slot = 0;
};

// Whether the persistent launch sweeps bucket b (all: the dependency queue).
bool persist_bucket(const BucketPlan &b, int prec, bool all) {
    if (prec != 0) return false;
    if (all) return b.N <= PERSIST_NMAX;
    return b.N <= PERSIST_SINGLE_NMAX && b.P.npass == 1;
}

long long persist_batch_families(int N) {
    const long long slot = 8LL << (N - 1);            // complex FP32 intermediate per family
    return std::max(1LL, (long long)PERSIST_SLOT_BYTES / slot);
}

// Segments in dependency order: two-pass buckets first (largest N first), each
// batch's strided items before the previous batch's row items; then the
// single-pass buckets. Marks the swept buckets (BucketPlan::persistent).
void persist_plan(std::vector<BucketPlan> &B, int prec, bool all, PersistLayout &L) {
    L = PersistLayout();
    L.buckets.resize(B.size());
    L.fm_off.assign(B.size(), 0);
    for (size_t bi = 0; bi < B.size(); ++bi) {
        B[bi].persistent = persist_bucket(B[bi], prec, all);
        if (!B[bi].persistent) continue;
        L.fm_off[bi] = L.fm_total;
        L.fm_total += (size_t)B[bi].idx.size() << B[bi].N;
    }
    auto push = [&](int kind, int bucket, int batch, int aux, long long count) {
        if (count <= 0) return;
        BatchSeg g;
        g.kind = kind; g.bucket = bucket; g.batch = batch; g.aux = aux; g.start = L.n_items; g.count = count;
        L.segs.push_back(g);
        L.n_items += count;
    };
    // a batch's row items follow the strided items of the PERSIST_AHEAD
    // batches after it, so that they rarely wait
    struct RowSeg { int bucket, batch; long long nf; };
    std::vector<RowSeg> pending;
    for (size_t bi = 0; bi < B.size(); ++bi) {
        const int N = B[bi].N;
        if (!B[bi].persistent || N <= PERSIST_SINGLE_NMAX) continue;
        L.dep = true;
        const long long fams = (long long)B[bi].idx.size() << N;
        const long long Bf = persist_batch_families(N);
        const int tiles = 1 << (N - 1 - 13);
        L.buckets[bi].first_batch = L.batches;
        L.tiles_slot = std::max(L.tiles_slot, (size_t)(Bf * tiles));
        for (long long fb = 0; fb < fams; fb += Bf) {
            const long long nf = std::min(Bf, fams - fb);
            const int groups = (int)((nf + PERSIST_FPC - 1) / PERSIST_FPC);
            const int k = L.batches++;
            push(BI_STRIDED, (int)bi, k, groups, (long long)tiles * groups);
            pending.push_back({(int)bi, k, nf});
            if ((int)pending.size() > PERSIST_AHEAD) {
                push(BI_ROW, pending.front().bucket, pending.front().batch, PERSIST_RPI,
                     (pending.front().nf + PERSIST_RPI - 1) / PERSIST_RPI);
                pending.erase(pending.begin());
            }
            L.need_str.push_back((unsigned)((long long)tiles * groups));
            L.need_row.push_back((unsigned)nf);
        }
    }
    for (const RowSeg &r : pending) push(BI_ROW, r.bucket, r.batch, PERSIST_RPI, (r.nf + PERSIST_RPI - 1) / PERSIST_RPI);
    for (size_t bi = 0; bi < B.size(); ++bi) {
        const int N = B[bi].N;
        if (!B[bi].persistent || N > PERSIST_SINGLE_NMAX) continue;
        const int M = N - 1;
        const int RB = M < 5 ? M : 5, TB = M - RB, G = TB >= 8 ? 1 : (256 >> TB);
        const long long fams = (long long)B[bi].idx.size() << N;
        push(BI_SINGLE, (int)bi, 0, G, (fams + G - 1) / G);
    }
}

// Device tables of the layout, pointing into the workspace.
void persist_tables(const std::vector<BucketPlan> &B, const BatchWS &w, float cand_thr, PersistLayout &L) {
    for (size_t bi = 0; bi < B.size(); ++bi) {
        const BucketPlan &b = B[bi];
        BatchBucket &k = L.buckets[bi];
        const int first_batch = k.first_batch;          // set by persist_plan
        memset(&k, 0, sizeof k);
        if (!b.persistent) continue;
        const int N = b.N;
        const long long fams = (long long)b.idx.size() << N;
        PassArgs a;
        memset(&a, 0, sizeof a);
        a.N = N;
        a.n = N - 1;
        a.slot_elems = 1LL << (N - 1);
        a.cand_thr = cand_thr;
        a.want_cand = 1;
        a.psi_list = w.psi_list + b.off;
        a.s_list = w.s_list + b.off;
        a.s_ptr = w.s_list + b.off;
        k.fm = w.fm_all + L.fm_off[bi];
        k.fam_total = fams;
        if (N > PERSIST_SINGLE_NMAX) {
            k.M = 13;
            k.K = N - 14;
            k.B = persist_batch_families(N);
            k.tiles_row = 1 << (N - 1 - 13);
            k.first_batch = first_batch;
            k.strided = a;
            k.strided.lo_g = 13;                // the strided rows are the packed bits 13 .. N - 2
            k.row = a;
            k.row.lo_g = 0;
        } else {
            k.M = N - 1;
            k.tiles_row = 1;
            k.single = a;
            k.single.fam_base = 0;
            k.single.n_fam = fams;
            k.single.fam_out = k.fm;
        }
    }
}


constexpr int BATCH_NORM_BLOCKS = 16;

struct BatchGraph {
    std::vector<int> shape;     // N of every slot, in slot order
    void *ws = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;
    int prec = 0;
    double eps = 0.0;           // nullity tolerance (sets the candidate threshold)
    std::vector<long long> plan;  // every bucket's tiling (plan_signature)
};

// The tiling a bucket's launch sequence was captured with: a cached graph is
// replayed only for the same plans (options and the autotuner's table can
// change them for the same batch shape).
std::vector<long long> plan_signature(const std::vector<BucketPlan> &B) {
    std::vector<long long> v;
    for (const BucketPlan &b : B) {
        v.push_back(b.persistent ? 1 : 0);
        v.insert(v.end(), {(long long)b.N, (long long)b.P.npass, (long long)b.P.M_last, b.P.B, b.P.tiles_last,
                           (long long)b.states_per_chunk});
        for (int i = 0; i < b.P.nstrided; ++i) v.insert(v.end(), {(long long)b.P.K[i], (long long)b.P.lo[i]});
    }
    return v;
}
std::mutex g_bgraph_mu;
std::vector<BatchGraph> g_bgraph;

void layout_batch(Arena &A, int count, std::vector<BucketPlan> &B, BatchWS &w, const PersistLayout *L = nullptr) {
    w.psi_list = A.take<const float2 *>(count);
    w.s_list = A.take<double>(count);
    w.norm_list = A.take<double>(count);
    w.npart = A.take<double>((size_t)count * BATCH_NORM_BLOCKS);
    w.totals = A.take<double>(TOT_N * (size_t)count);
    w.state_count = A.take<unsigned long long>(count);
    w.nflag = A.take<unsigned long long>(B.size());
    size_t fm_n = 0, tiles_n = 0, inter_b = 0, inter64_b = 0, counts_n = 0;
    for (auto &b : B) {
        const long long fams = (long long)b.idx.size() << b.N;
        b.flags = A.take<unsigned long long>((size_t)fams);
        b.flag_cap = fams;
        counts_n = std::max(counts_n, (size_t)fams);
        if (b.persistent) {
            // the nullity recount of the flagged families still runs through
            // the chunked intermediates (its FP32 candidate pass and the FP64
            // transform)
            if (b.P.npass > 1) inter_b = std::max(inter_b, b.P.slot_bytes * (size_t)b.P.B);
            if (b.P64.npass > 1) inter64_b = std::max(inter64_b, b.P64.slot_bytes * (size_t)b.P64.B);
            continue;
        }
        const long long chunk = (long long)b.states_per_chunk << b.N;
        fm_n = std::max(fm_n, (size_t)chunk);
        if (b.P.npass == 1) tiles_n = std::max(tiles_n, (size_t)chunk);
        else {
            tiles_n = std::max(tiles_n, (size_t)(b.P.B * b.P.tiles_last));
            inter_b = std::max(inter_b, b.P.slot_bytes * (size_t)b.P.B);
        }
        if (b.P64.npass > 1) inter64_b = std::max(inter64_b, b.P64.slot_bytes * (size_t)b.P64.B);
        counts_n = std::max(counts_n, (size_t)fams);
    }
    w.fm = A.take<FamMoments>(fm_n);
    w.tiles = A.take<TilePartial>(tiles_n);
    w.inter = inter_b ? (void *)A.take<char>(inter_b) : nullptr;
    w.inter64 = inter64_b ? (void *)A.take<char>(inter64_b) : nullptr;
    w.counts = A.take<unsigned long long>(counts_n);
    w.fm_all = nullptr;
    w.pbuckets = nullptr;
    w.psegs = nullptr;
    w.next = nullptr;
    w.need = w.done = nullptr;
    w.abort_flag = w.err = nullptr;
    w.ring = nullptr;
    w.ring_tiles = nullptr;
    if (L && L->n_items) {
        w.fm_all = A.take<FamMoments>(L->fm_total);
        w.pbuckets = A.take<BatchBucket>(L->buckets.size());
        w.psegs = A.take<BatchSeg>(L->segs.size());
        w.next = A.take<unsigned long long>(1);
        if (L->dep) {
            w.need = A.take<unsigned>(2 * (size_t)L->batches + 2);
            w.done = A.take<unsigned>(2 * (size_t)L->batches + 2);
            w.abort_flag = A.take<int>(1);
            w.err = A.take<int>(1);
            w.ring = (void *)A.take<char>((size_t)PERSIST_RING * PERSIST_SLOT_BYTES);
            w.ring_tiles = A.take<TilePartial>((size_t)PERSIST_RING * L->tiles_slot + 1);
        }
    }
    layout_null(A, (long long)counts_n, w.nw);
    w.nw.counts = w.counts;
    w.nw.inter = w.inter;
    w.nw.inter64 = w.inter64;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// The main launch sequence (captured into the graph): per-bucket norms, one
// persistent launch over every family of the buckets it sweeps (k_batch.cu)
// with their per-state totals, then every other bucket chunk by chunk. The
// tables the persistent launch reads (L) are uploaded before every run.
sre_status batch_main(const std::vector<BucketPlan> &B, const BatchWS &w, const PersistLayout &L, int count, int prec,
                      float cand_thr, cudaStream_t st) {
    CK(cudaMemsetAsync(w.nflag, 0, sizeof(unsigned long long) * B.size(), st));
    CK(cudaMemsetAsync(w.state_count, 0, sizeof(unsigned long long) * count, st));
    for (size_t bi = 0; bi < B.size(); ++bi) {
        const BucketPlan &b = B[bi];
        CK(launch_norm2_multi(w.psi_list + b.off, (int)b.idx.size(), b.N, w.npart, BATCH_NORM_BLOCKS,
                              w.norm_list + b.off, w.s_list + b.off, st));
        count_launches(2);
    }
    if (L.n_items > 0) {
        CK(cudaMemsetAsync(w.next, 0, sizeof(unsigned long long), st));
        BatchQueue q;
        memset(&q, 0, sizeof q);
        q.segs = w.psegs;
        q.n_segs = (int)L.segs.size();
        q.n_items = L.n_items;
        q.buckets = w.pbuckets;
        q.next = w.next;
        if (L.dep) {
            CK(cudaMemsetAsync(w.done, 0, sizeof(unsigned) * (2 * (size_t)L.batches + 2), st));
            CK(cudaMemsetAsync(w.abort_flag, 0, sizeof(int), st));
            CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
            q.done_str = w.done;
            q.done_row = w.done + L.batches;
            q.need_str = w.need;
            q.need_row = w.need + L.batches;
            q.inter = w.ring;
            q.inter_slot_bytes = PERSIST_SLOT_BYTES;
            q.tiles = w.ring_tiles;
            q.tiles_slot = L.tiles_slot;
            q.ring = PERSIST_RING;
            q.fpc = PERSIST_FPC;
            q.err = w.err;
            q.abort_flag = w.abort_flag;
        }
        CK(launch_batch_persistent(q, L.dep, 2 * sm_count(), st));
        count_launches(1);
        for (size_t bi = 0; bi < B.size(); ++bi) {
            const BucketPlan &b = B[bi];
            if (!b.persistent) continue;
            CK(launch_state_totals(w.fm_all + L.fm_off[bi], 0, b.N, 0, (int)b.idx.size(),
                                   w.totals + TOT_N * (size_t)b.off, b.flags, w.nflag + bi, st));
            count_launches(1);
        }
    }
    for (size_t bi = 0; bi < B.size(); ++bi) {
        const BucketPlan &b = B[bi];
        if (b.persistent) continue;
        const int ns = (int)b.idx.size();
        PassArgs a = base_args(b.P, nullptr, w.s_list + b.off);
        a.precision = prec;
        a.cand_thr = cand_thr;
        a.psi_list = w.psi_list + b.off;
        a.s_list = w.s_list + b.off;
        a.tile_out = w.tiles;
        for (int c0 = 0; c0 < ns; c0 += b.states_per_chunk) {
            const int c1 = std::min(ns, c0 + b.states_per_chunk);
            const long long f0 = (long long)c0 << b.N, f1 = (long long)c1 << b.N;
            const long long step = b.P.npass > 1 ? b.P.B : (f1 - f0);
            for (long long fb = f0; fb < f1; fb += step) {
                const long long nf = std::min(step, f1 - fb);
                PassArgs c = a;
                c.fam_base = fb;
                c.n_fam = nf;
                CS(run_transform(b.P, c, SRC_PSI_FAMILY, DST_MOMENTS, w.inter, st));
                CK(launch_fam_reduce(w.tiles, nf, (int)b.P.tiles_last, nullptr, fb, b.N, b.P.M_last, b.P.M_last,
                                     w.fm, fb - f0, nullptr, 0, st));
                count_launches(1);
            }
            CK(launch_state_totals(w.fm, f0, b.N, c0, c1 - c0, w.totals + TOT_N * (size_t)b.off, b.flags,
                                   w.nflag + bi, st));
            count_launches(1);
        }
    }
    return SRE_OK;
}

sre_status batched_impl(const void *const *psi_ptrs, const int *Ns, int count, const sre_opts &o,
                        cudaStream_t st, sre_result *out) {
    // buckets by N, largest first
    std::vector<BucketPlan> B;
    {
        std::vector<std::vector<int>> by(21);
        for (int i = 0; i < count; ++i) by[Ns[i]].push_back(i);
        int off = 0;
        for (int N = 20; N >= 1; --N) {
            if (by[N].empty()) continue;
            BucketPlan b;
            b.N = N;
            b.idx = by[N];
            b.off = off;
            off += (int)b.idx.size();
            CS(plan_for_tuned(N, &o, 32, b.P));
            CS(plan_for(N, nullptr, 64, b.P64));
            b.states_per_chunk = (int)std::max(1LL, BATCH_CHUNK_FAMILIES >> N);
            b.flags = nullptr;
            b.flag_cap = 0;
            b.persistent = false;
            B.push_back(b);
        }
    }
    // one persistent launch over the single-pass buckets of the FP32 sweep
    // (with opts.batch_queue: over every bucket)
    PersistLayout L;
    persist_plan(B, prec_code(o), o.batch_queue != 0, L);
    Arena dry(nullptr);
    BatchWS w;
    layout_batch(dry, count, B, w, &L);
    void *base = nullptr;
    CS(own_workspace(dry.off, &base));
    Arena A(base);
    layout_batch(A, count, B, w, &L);
    if (L.n_items > 0) {
        persist_tables(B, w, cand_threshold(o.eps_null), L);
        CK(cudaMemcpyAsync(w.pbuckets, L.buckets.data(), sizeof(BatchBucket) * L.buckets.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(w.psegs, L.segs.data(), sizeof(BatchSeg) * L.segs.size(), cudaMemcpyHostToDevice, st));
        if (L.dep) {
            CK(cudaMemcpyAsync(w.need, L.need_str.data(), sizeof(unsigned) * L.batches, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(w.need + L.batches, L.need_row.data(), sizeof(unsigned) * L.batches,
                               cudaMemcpyHostToDevice, st));
        }
    }

    // psi pointers in slot (bucket) order
    std::vector<const float2 *> hp(count);
    std::vector<int> shape(count);
    for (const auto &b : B)
        for (size_t k = 0; k < b.idx.size(); ++k) {
            hp[b.off + k] = (const float2 *)psi_ptrs[b.idx[k]];
            shape[b.off + k] = b.N;
        }
    CK(cudaMemcpyAsync((void *)w.psi_list, hp.data(), sizeof(const float2 *) * count, cudaMemcpyHostToDevice, st));

    // main sequence: replay a cached graph of the same shape on the same workspace, else capture one
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;
    const std::vector<long long> sig = plan_signature(B);
    {
        std::lock_guard<std::mutex> lk(g_bgraph_mu);
        for (auto &g : g_bgraph)
            if (g.ws == base && g.shape == shape && g.prec == prec_code(o) && g.eps == o.eps_null && g.plan == sig) {
                exec = g.exec;
                kernels = g.kernels;
                break;
            }
    }
    if (!exec) {
        cudaStream_t cap;
        CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { cudaStreamDestroy(cap); return fail(SRE_ECUDA, "capture: %s", cudaGetErrorString(e)); }
        const unsigned long long l0 = g_launches.load();
        sre_status s1 = batch_main(B, w, L, count, prec_code(o), cand_threshold(o.eps_null), cap);
        e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (s1 != SRE_OK) { if (e == cudaSuccess) cudaGraphDestroy(graph); return s1; }
        if (e != cudaSuccess) return fail(SRE_ECUDA, "end capture: %s", cudaGetErrorString(e));
        kernels = g_launches.load() - l0;
        g_launches.fetch_sub(kernels);   // counted when the graph runs
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(SRE_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        std::lock_guard<std::mutex> lk(g_bgraph_mu);
        BatchGraph g;
        g.shape = shape;
        g.ws = base;
        g.exec = exec;
        g.kernels = kernels;
        g.prec = prec_code(o);
        g.eps = o.eps_null;
        g.plan = sig;
        g_bgraph.push_back(g);
    }
    CK(cudaGraphLaunch(exec, st));
    count_launches(kernels);

    std::vector<unsigned long long> nflag(B.size());
    CK(cudaMemcpyAsync(nflag.data(), w.nflag, sizeof(unsigned long long) * B.size(), cudaMemcpyDeviceToHost, st));
    int perr = 0;
    if (L.dep) CK(cudaMemcpyAsync(&perr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (perr & SRE_ERR_TIMEOUT) return fail(SRE_ETIMEOUT, "a bounded wait of the persistent batched sweep expired");

    // FP64 recount of the candidate families, per bucket
    for (size_t bi = 0; bi < B.size(); ++bi) {
        const BucketPlan &b = B[bi];
        const long long nf = (long long)nflag[bi];
        if (nf <= 0) continue;
        PassArgs a32 = base_args(b.P, nullptr, w.s_list + b.off), a64 = base_args(b.P64, nullptr, w.s_list + b.off);
        a32.psi_list = a64.psi_list = w.psi_list + b.off;
        a32.s_list = a64.s_list = w.s_list + b.off;
        long long no = 0;
        CS(null_recount(b.P, b.P64, a32, a64, b.flags, nf, o.eps_null, w.nw, st, &no));
        CK(launch_count_scatter(b.flags, w.counts, nf, b.N, w.state_count + b.off, st));
        count_launches(1);
        if (no > 0) {
            CK(launch_count_scatter(w.nw.ovf, w.nw.counts2, no, b.N, w.state_count + b.off, st));
            count_launches(1);
        }
    }
    std::vector<double> tot(TOT_N * (size_t)count), nrm(count);
    std::vector<unsigned long long> cnt(count);
    CK(cudaMemcpyAsync(tot.data(), w.totals, sizeof(double) * TOT_N * count, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(nrm.data(), w.norm_list, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(cnt.data(), w.state_count, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool zero = false;
    for (const auto &b : B)
        for (size_t k = 0; k < b.idx.size(); ++k) {
            const int slot = b.off + (int)k;
            sre_result *r = out + b.idx[k];
            init_result(r);
            finalize_exact(&tot[TOT_N * (size_t)slot], b.N, r);
            r->n_families = 1LL << b.N;
            r->n_passes = b.P.npass;
            if (!(nrm[slot] > 0.0)) { zero = true; continue; }
            nullity_from_count((long long)cnt[slot], b.N, r);   // nullity -1 if not a power of two
        }
    if (zero) return fail(SRE_EZERO, "a state of the batch has zero norm");
    return SRE_OK;
}

// --------------------------------------------------------------- autotuner
// Times the family-transform launch sequence of every admissible plan for N
// on the caller's state and keeps the fastest (radix, tile, x_batch).
sre_status autotune_impl(const void *psi, int N, cudaStream_t st, sre_opts *best) {
    sre_default_opts(best);
    Plan P0;
    CS(plan_for(N, nullptr, 32, P0));
    if (P0.npass == 1) return SRE_OK;   // nothing to choose
    struct Cand { int radix, tile, xb; };
    std::vector<Cand> cands;
    for (int r = F32_ROW_MMIN; r <= F32_ROW_MMAX; ++r)
        for (int t : {0, 8})
            for (int xb : {0, 8})
                cands.push_back({r, t, xb});
    double best_rate = -1.0;
    const long long d = 1LL << N;
    for (const Cand &c : cands) {
        sre_opts q;
        sre_default_opts(&q);
        q.radix_log2 = c.radix;
        q.tile_log2 = c.tile;
        q.x_batch = c.xb;
        Plan P;
        if (plan_for(N, &q, 32, P) != SRE_OK) continue;
        const long long fams = std::min(d, std::max(P.B * 4, 64LL));
        Arena dry(nullptr);
        McWS w;
        layout_mc(dry, P, SRE_MC_UNIFORM, fams, 1, w);
        void *base = nullptr;
        CS(own_workspace(dry.off, &base));
        Arena A(base);
        layout_mc(A, P, SRE_MC_UNIFORM, fams, 1, w);
        CK(launch_norm2((const float2 *)psi, N, w.scal, w.npart, st));
        count_launches(2);
        PassArgs a = base_args(P, psi, w.scal);
        a.tile_out = w.tiles;
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {   // rep 0 warms up
            CK(cudaEventRecord(e0, st));
            for (long long fb = 0; fb < fams; fb += P.B) {
                PassArgs b = a;
                b.fam_base = fb;
                b.n_fam = std::min(P.B, fams - fb);
                CS(run_transform(P, b, SRC_PSI_FAMILY, DST_MOMENTS, w.inter, st));
            }
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(&ms, e0, e1));
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const double rate = (double)fams * (double)d / (ms * 1e-3);
        if (rate > best_rate) {
            best_rate = rate;
            best->radix_log2 = c.radix;
            best->tile_log2 = c.tile;
            best->x_batch = c.xb;
        }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    g_tune[N].radix = best->radix_log2;
    g_tune[N].tile = best->tile_log2;
    g_tune[N].xbatch = best->x_batch;
    g_tune[N].valid = true;
    tune_save_locked();
    return SRE_OK;
}

// Gates are grouped into blocks of at most GATE_BLOCK_Q qubits (qubits
// 0..GATE_BLOCK_LOW-1 always included), each applied in one pass over psi in
// shared memory. Grouping follows the circuit's dependencies, not only its
// list order: a gate joins the current block once every earlier gate on its
// qubits has been applied (in an earlier block or earlier in this one), the
// cheapest such gate first (fewest qubits added, then the earliest), until no
// ready gate fits. Gates on disjoint qubits commute, so any such order
// applies the same unitary. Rows: op, q0, q1 (global qubits; q1 used by CNOT
// and U2); mats_host: 32 floats per row (U2 rows only; NULL when there are none).
sre_status run_gate_list(void *psi, int N, const std::vector<GateRow> &in_rows, const float *mats_host,
                         cudaStream_t st) {
    const long long n_gates = (long long)in_rows.size();
    if (n_gates == 0) return SRE_OK;
    const int low = N < GATE_BLOCK_LOW ? N : GATE_BLOCK_LOW;
    const int qmax = N < GATE_BLOCK_Q ? N : GATE_BLOCK_Q;
    auto two = [](const GateRow &G) { return G.op == SRE_GATE_CNOT || G.op == GATE_OP_U2; };
    std::vector<std::vector<long long>> qlist(N);
    for (long long g = 0; g < n_gates; ++g) {
        qlist[in_rows[g].q0].push_back(g);
        if (two(in_rows[g])) qlist[in_rows[g].q1].push_back(g);
    }
    std::vector<size_t> ptr(N, 0);
    auto ready = [&](long long g) {
        const GateRow &G = in_rows[g];
        if (ptr[G.q0] >= qlist[G.q0].size() || qlist[G.q0][ptr[G.q0]] != g) return false;
        return !two(G) || (ptr[G.q1] < qlist[G.q1].size() && qlist[G.q1][ptr[G.q1]] == g);
    };
    std::vector<int> blocks;
    std::vector<unsigned char> bq;
    std::vector<GateRow> rows;
    std::vector<float> mats;
    rows.reserve(n_gates);
    if (mats_host) mats.reserve(32 * (size_t)n_gates);
    long long ndone = 0;
    while (ndone < n_gates) {
        bool in[64] = {false};
        int cnt = 0;
        for (int q = 0; q < low; ++q) { in[q] = true; ++cnt; }
        std::vector<long long> blk;
        for (;;) {
            if (mats_host && (int)blk.size() >= GATE_BLOCK_MAX_U2) break;
            long long best = -1;
            int best_new = 3;
            for (int q = 0; q < N; ++q) {
                if (ptr[q] >= qlist[q].size()) continue;
                const long long g = qlist[q][ptr[q]];
                if (!ready(g)) continue;
                const GateRow &G = in_rows[g];
                const int add = (!in[G.q0]) + (two(G) && !in[G.q1] ? 1 : 0);
                if (cnt + add > qmax) continue;
                if (add < best_new || (add == best_new && g < best)) { best = g; best_new = add; }
            }
            if (best < 0) break;
            const GateRow &G = in_rows[best];
            if (!in[G.q0]) { in[G.q0] = true; ++cnt; }
            if (two(G) && !in[G.q1]) { in[G.q1] = true; ++cnt; }
            ++ptr[G.q0];
            if (two(G)) ++ptr[G.q1];
            blk.push_back(best);
        }
        unsigned char loc[64];
        unsigned char list[GATE_BLOCK_Q];
        int m = 0;
        for (int q = 0; q < N; ++q)
            if (in[q]) { loc[q] = (unsigned char)m; list[m++] = (unsigned char)q; }
        for (int i = m; i < GATE_BLOCK_Q; ++i) list[i] = 255;
        blocks.push_back((int)rows.size());
        blocks.push_back((int)blk.size());
        for (long long g : blk) {
            GateRow r;
            r.op = in_rows[g].op;
            r.q0 = loc[in_rows[g].q0];
            r.q1 = two(in_rows[g]) ? loc[in_rows[g].q1] : 0;
            rows.push_back(r);
            if (mats_host) mats.insert(mats.end(), mats_host + 32 * g, mats_host + 32 * (g + 1));
        }
        bq.insert(bq.end(), list, list + GATE_BLOCK_Q);
        ndone += (long long)blk.size();
        if (blk.empty()) return fail(SRE_EINVAL, "gate planner made no progress");
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    GateRow *dg = nullptr;
    float2 *dm = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        if ((int)g_gatebuf.size() <= dev) g_gatebuf.resize(dev + 1);
        DevBuf &b = g_gatebuf[dev];
        const size_t rows_bytes = (sizeof(GateRow) * (size_t)n_gates + 255) & ~(size_t)255;
        const size_t need = rows_bytes + (mats_host ? sizeof(float2) * 16 * (size_t)n_gates : 0);
        if (b.n < need) {
            if (b.p) CK(cudaFree(b.p));
            b.p = nullptr;
            b.n = 0;
            cudaError_t e = cudaMalloc(&b.p, need);
            g_allocs.fetch_add(1, std::memory_order_relaxed);
            if (e != cudaSuccess) return fail(SRE_ENOMEM, "gate buffer: %s", cudaGetErrorString(e));
            b.n = need;
        }
        dg = (GateRow *)b.p;
        if (mats_host) dm = (float2 *)((char *)b.p + rows_bytes);
    }
    CK(cudaMemcpyAsync(dg, rows.data(), sizeof(GateRow) * (size_t)n_gates, cudaMemcpyHostToDevice, st));
    if (mats_host)
        CK(cudaMemcpyAsync(dm, mats.data(), sizeof(float2) * 16 * (size_t)n_gates, cudaMemcpyHostToDevice, st));
    CK(launch_gate_blocks((float2 *)psi, N, dg, dm, blocks.data(), (int)(blocks.size() / 2), bq.data(), st));
    count_launches(blocks.size() / 2);
    CK(cudaStreamSynchronize(st));
    return SRE_OK;
}

// ------------------------------------------------------ mixed states
struct MixedWS {
    double *scal, *npart, *epart, *etot;
    float2 *C;
    TilePartial *tiles;
    FamMoments *fm;
    void *planes;      // BF16 split planes of Psi for the tensor-core Gram kernel (one K chunk)
    int *err;          // device error word
};

void layout_mixed(Arena &A, int N, int NA, MixedWS &w) {
    const unsigned long long dA = 1ULL << NA;
    w.scal = A.take<double>(SCAL_N);
    w.npart = A.take<double>(NORM_BLOCKS);
    w.epart = A.take<double>(6 * EXACT_PARTS);
    w.etot = A.take<double>(8);
    w.C = A.take<float2>(dA * dA);
    w.tiles = A.take<TilePartial>(dA);
    w.fm = A.take<FamMoments>(dA);
    w.planes = A.take<unsigned char>(gram_plane_bytes(N, NA));
    w.err = A.take<int>(1);
}

// SRE of the reduced state on the first N_A qubits (SM, mixed states):
// C = Psi Psi^H on the tensor cores (Psi = psi viewed column-major d_A x d_B;
// k_gram.cu), then every family x_A of the N_A-qubit system through the
// single-pass transform with the h(a) = C[a][a ^ x_A] prologue and the fused
// moments, then the fixed-order FP64 totals; Eq. Msre-mixed on the host.
sre_status mixed_impl(const void *psi, int N, int NA, void *ws, size_t ws_bytes, cudaStream_t st,
                      sre_mixed_result *out) {
    Arena dry(nullptr);
    MixedWS w;
    layout_mixed(dry, N, NA, w);
    void *base = nullptr;
    CS(resolve_workspace(ws, ws_bytes, dry.off, &base));
    Arena A(base);
    layout_mixed(A, N, NA, w);
    const unsigned long long dA = 1ULL << NA;
    CK(launch_norm2((const float2 *)psi, N, w.scal, w.npart, st));
    count_launches(2);
    CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    int gl = 0;
    cudaError_t ge = launch_gram((const float2 *)psi, N, NA, w.C, w.planes, w.err, &gl, st);
    count_launches(gl);
    if (ge != cudaSuccess) return fail(SRE_ECUDA, "Gram matrix (N=%d, N_A=%d): %s", N, NA, cudaGetErrorString(ge));
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.N = NA;
    a.n = NA - 1;
    a.slot_elems = 1LL << (NA - 1);
    a.range_log2 = NA - 1;
    a.s_ptr = w.scal + SCAL_S;
    a.tile_out = w.tiles;
    a.cand_thr = 1.0f;
    a.gram = w.C;
    a.gram_ld = (long long)dA;
    a.fam_base = 0;
    a.n_fam = (long long)dA;
    cudaError_t e = launch_f32_single(NA - 1, SRC_GRAM, DST_MOMENTS, a, st);
    if (e != cudaSuccess) return fail(SRE_ECUDA, "mixed-state transform (N_A=%d): %s", NA, cudaGetErrorString(e));
    count_launches(1);
    CK(launch_fam_reduce(w.tiles, (long long)dA, 1, nullptr, 0, NA, NA - 1, NA - 1, w.fm, 0, nullptr, 0, st));
    count_launches(1);
    unsigned long long *no_flags = nullptr;
    CK(launch_exact_totals(w.fm, (long long)dA, w.epart, EXACT_PARTS, w.etot, no_flags, nullptr, st));
    count_launches(2);
    double T[TOT_N + 1];
    CK(cudaMemcpyAsync(T, w.etot, TOT_N * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(T + TOT_N, w.scal + SCAL_NORM2, sizeof(double), cudaMemcpyDeviceToHost, st));
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr & SRE_ERR_TIMEOUT) return fail(SRE_ETIMEOUT, "Gram matrix: a bounded wait ran out");
    if (!(T[TOT_N] > 0.0)) return fail(SRE_EZERO, "psi has zero norm");
    memset(out, 0, sizeof *out);
    const double da = (double)dA;
    for (int i = 0; i < 4; ++i) out->W[i] = T[i];
    out->S2 = -std::log2(T[0] / da);
    out->M[1] = -std::log2(T[1] / (da * da)) - NA - out->S2;
    out->M[2] = -0.5 * std::log2(T[2] / (da * da * da)) - NA - out->S2;
    // a-priori FP32 rounding estimate, as for the pure sweep over N_A + log2 d_B sums
    const double ec = (N + 2) * std::ldexp(1.0, -24);
    out->M[0] = std::fabs(out->S2) <= 64.0 * ec ? -T[3] / da : std::nan("");
    out->err_M[0] = 2.0 * ec * (N + 2);
    out->err_M[1] = 4.0 * ec / std::log(2.0) + 2.0 * ec / std::log(2.0);
    out->err_M[2] = 6.0 * ec / (2.0 * std::log(2.0)) + 2.0 * ec / std::log(2.0);
    out->N_A = NA;
    return SRE_OK;
}

} // namespace

namespace sre {
// error message of the calling thread for entry points in other units
void set_error_message(const char *msg) { g_err = msg; }
}

// =================================================================== C ABI
extern "C" {

const char *sre_version(void) { return "sre-gb300 0.1 (sm_103a)"; }

const char *sre_last_error(void) { return g_err.c_str(); }

void sre_default_opts(sre_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = SRE_FP32_SIMT;
    o->eps_null = 1e-6;
}

sre_status sre_make_plan(int N, const sre_opts *opts, sre_plan *plan) {
    if (!plan) return fail(SRE_EINVAL, "plan is NULL");
    if (N < 1 || N > 32) return fail(SRE_EINVAL, "N=%d outside 1..32", N);
    sre_opts o;
    CS(check_opts(opts, o));
    Plan P;
    CS(plan_for_tuned(N, &o, 32, P));
    memset(plan, 0, sizeof *plan);
    plan->N = N;
    plan->n_bits = P.n;
    plan->n_passes = P.npass;
    for (int i = 0; i < P.nstrided; ++i) { plan->pass_lo[i] = P.lo[i]; plan->pass_bits[i] = P.K[i]; }
    plan->pass_lo[P.npass - 1] = 0;
    plan->pass_bits[P.npass - 1] = P.M_last;
    plan->x_batch = (int)(P.B > 0x7fffffff ? 0x7fffffff : P.B);
    plan->range_log2 = P.RL;
    if (N <= 26) {
        size_t b = 0;
        if (sre_workspace_bytes(N, -1, 0, 0, &o, &b) == SRE_OK) plan->workspace_exact = b;
    }
    return SRE_OK;
}

sre_status sre_workspace_bytes(int N, int mode, long long n_x, int z_per_x, const sre_opts *opts, size_t *bytes) {
    if (!bytes) return fail(SRE_EINVAL, "bytes is NULL");
    sre_opts o;
    CS(check_opts(opts, o));
    Plan P;
    if (mode == -1) {
        if (N < 1 || N > 26) return fail(SRE_EINVAL, "exact: N=%d outside 1..26", N);
        Plan P64;
        CS(plan_for_tuned(N, &o, 32, P));
        CS(plan_for(N, nullptr, 64, P64));
        Arena A(nullptr);
        ExactWS w;
        layout_exact(A, P, P64, w);
        *bytes = A.off;
        return SRE_OK;
    }
    if (mode != SRE_MC_UNIFORM && mode != SRE_MC_MARGINAL) return fail(SRE_EINVAL, "unknown mode %d", mode);
    if (N < 2 || N > 30) return fail(SRE_EINVAL, "mc: N=%d outside 2..30", N);
    if (n_x < 2 || (mode == SRE_MC_MARGINAL && z_per_x < 1)) return fail(SRE_EINVAL, "n_x >= 2 and z_per_x >= 1 required");
    CS(plan_for_tuned(N, &o, 32, P));
    Arena A(nullptr);
    McWS w;
    layout_mc(A, P, mode, n_x, z_per_x, w);
    *bytes = A.off;
    return SRE_OK;
}

sre_status sre_release_workspace(void) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if ((int)g_ws.size() > dev && g_ws[dev].p) {
        CK(cudaFree(g_ws[dev].p));
        g_ws[dev] = DevWS();
    }
    if ((int)g_gatebuf.size() > dev && g_gatebuf[dev].p) {
        CK(cudaFree(g_gatebuf[dev].p));
        g_gatebuf[dev] = DevBuf();
    }
    return SRE_OK;
}

sre_status sre_norm2(const void *psi, int N, double *norm2_host, void *stream) {
    CS(check_psi(psi, N, 1, 32));
    if (!norm2_host) return fail(SRE_EINVAL, "norm2_host is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    void *base = nullptr;
    CS(own_workspace(sizeof(double) * (SCAL_N + NORM_BLOCKS) + 1024, &base));
    double *scal = (double *)base;
    double *part = scal + SCAL_N;
    CK(launch_norm2((const float2 *)psi, N, scal, part, st));
    count_launches(2);
    CK(cudaMemcpyAsync(norm2_host, scal + SCAL_NORM2, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SRE_OK;
}

sre_status sre_exact(const void *psi, int N, const sre_opts *opts, void *workspace, size_t workspace_bytes,
                     void *stream, sre_result *out) {
    CS(check_psi(psi, N, 1, 26));
    if (!out) return fail(SRE_EINVAL, "out is NULL");
    sre_opts o;
    CS(check_opts(opts, o));
    return exact_impl(psi, N, o, workspace, workspace_bytes, (cudaStream_t)stream, out);
}

sre_status sre_exact_batched(const void *const *psi_ptrs, const int *Ns, int count, const sre_opts *opts,
                             void *workspace, size_t workspace_bytes, void *stream, sre_result *out) {
    if (count < 0 || (count > 0 && (!psi_ptrs || !Ns || !out))) return fail(SRE_EINVAL, "bad batch arguments");
    sre_opts o;
    CS(check_opts(opts, o));
    for (int i = 0; i < count; ++i) CS(check_psi(psi_ptrs[i], Ns[i], 1, 20));
    if (workspace) return fail(SRE_ENOTSUP, "sre_exact_batched uses the library workspace (pass NULL)");
    (void)workspace_bytes;
    if (count == 0) return SRE_OK;
    return batched_impl(psi_ptrs, Ns, count, o, (cudaStream_t)stream, out);
}

sre_status sre_autotune(const void *psi, int N, void *stream, sre_opts *best) {
    CS(check_psi(psi, N, 2, 26));
    if (!best) return fail(SRE_EINVAL, "best is NULL");
    return autotune_impl(psi, N, (cudaStream_t)stream, best);
}

sre_status sre_autotune_clear(int N) {
    if (N < 0 || N > 32) return fail(SRE_EINVAL, "N=%d outside 0..32", N);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    for (int n = 1; n <= 32; ++n)
        if (N == 0 || n == N) g_tune[n] = TuneEntry();
    tune_save_locked();
    return SRE_OK;
}

sre_status sre_mc(const void *psi, int N, int mode, long long n_x, int z_per_x, unsigned long long seed,
                  unsigned long long counter0, const sre_opts *opts, void *workspace, size_t workspace_bytes,
                  void *stream, sre_result *out, unsigned long long *xs_dev, unsigned long long *zs_dev,
                  float *c_dev) {
    CS(check_psi(psi, N, 2, 30));
    if (!out) return fail(SRE_EINVAL, "out is NULL");
    if (mode != SRE_MC_UNIFORM && mode != SRE_MC_MARGINAL) return fail(SRE_EINVAL, "unknown mode %d", mode);
    if (n_x < 2) return fail(SRE_EINVAL, "n_x must be >= 2");
    if (mode == SRE_MC_MARGINAL && (z_per_x < 1 || z_per_x > (1 << 20)))
        return fail(SRE_EINVAL, "z_per_x must be in 1..2^20");
    if (mode == SRE_MC_UNIFORM) z_per_x = 1;
    sre_opts o;
    CS(check_opts(opts, o));
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    CS(plan_for_tuned(N, &o, 32, P));
    Arena dry(nullptr);
    McWS w;
    layout_mc(dry, P, mode, n_x, z_per_x, w);
    void *base = nullptr;
    CS(resolve_workspace(workspace, workspace_bytes, dry.off, &base));
    Arena A(base);
    layout_mc(A, P, mode, n_x, z_per_x, w);
    const bool marg = mode == SRE_MC_MARGINAL;
    const unsigned long long d = 1ULL << N;

    CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    CK(launch_norm2((const float2 *)psi, N, w.scal, w.npart, st));
    count_launches(2);
    if (marg) {
        CS(run_marginal(psi, N, w.scal, w.p, w.mwork, st));
        CK(launch_scan(w.p, d, w.p, w.bsum, st));
        count_launches(3);
    }
    CK(launch_draw_x(w.p, N, n_x, marg ? 1 : 0, seed, counter0, w.xs, st));
    count_launches(1);
    // Multi-pass plans process the families in an order that lets the
    // families of one launch share psi in L2: by the top bit j of x (the same
    // rows b for every family with that j), then by x's bits over the first
    // strided pass's tile index (partner tile = tile ^ those bits, so the
    // partner tiles of a launch span a few aligned blocks), then by index.
    // Each family keeps its own index for its moments, draw stream and
    // outputs, so no result depends on the order.
    const unsigned long long *xs_run = w.xs, *perm = nullptr;
    if (P.npass > 1) {
        std::vector<unsigned long long> hx((size_t)n_x), order((size_t)n_x), hxo((size_t)n_x);
        CK(cudaMemcpyAsync(hx.data(), w.xs, sizeof(unsigned long long) * (size_t)n_x, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const int cb = P.ms[0] - P.K[0], tb = P.lo[0] - cb;
        auto key = [&](unsigned long long x) {
            const unsigned long long j = x ? (unsigned long long)(63 - __builtin_clzll(x)) : 0ULL;
            return (j << 40) | ((x >> cb) & ((1ULL << tb) - 1ULL));
        };
        for (long long i = 0; i < n_x; ++i) order[(size_t)i] = (unsigned long long)i;
        std::sort(order.begin(), order.end(), [&](unsigned long long p, unsigned long long q) {
            const unsigned long long kp = key(hx[p]), kq = key(hx[q]);
            return kp != kq ? kp < kq : p < q;
        });
        for (long long i = 0; i < n_x; ++i) hxo[(size_t)i] = hx[order[(size_t)i]];
        CK(cudaMemcpyAsync(w.xs_ord, hxo.data(), sizeof(unsigned long long) * (size_t)n_x, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(w.perm, order.data(), sizeof(unsigned long long) * (size_t)n_x, cudaMemcpyHostToDevice,
                           st));
        CK(cudaStreamSynchronize(st));   // the host vectors go out of scope
        xs_run = w.xs_ord;
        perm = w.perm;
    }

    PassArgs a = base_args(P, psi, w.scal);
    a.precision = prec_code(o);
    a.xs = xs_run;
    a.tile_out = w.tiles;
    a.want_ranges = marg ? 1 : 0;
    a.want_cand = 0;                 // the estimators need no nullity candidates
    a.err_flag = w.err;
    a.rw_out = w.Wf;
    a.rw_stride = 1LL << (N - P.RL);
    const long long step = P.B < n_x ? P.B : n_x;
    const long long nr = 1LL << (N - P.RL);
    const bool fine = fine_ranges(P);
    bool timing;
    {
        std::lock_guard<std::mutex> lk(g_timing_mu);
        timing = g_timing_on;
    }
    PassTimer T;
    if (timing) timing_bytes(P, step);
    for (long long fb = 0; fb < n_x; fb += step) {
        const long long nf = n_x - fb < step ? n_x - fb : step;
        PassArgs b = a;
        b.fam_base = fb;
        b.n_fam = nf;
        // a last pass that adds two warps' sums into each range needs zeroed rows
        if (marg && fine && f32_row_ranges_accumulate(P.M_last))
            CK(cudaMemsetAsync(w.Wf, 0, sizeof(float) * (size_t)nf * (size_t)nr, st));
        CS(run_transform(P, b, SRC_PSI_FAMILY, DST_MOMENTS, w.inter, st, (timing && nf == step) ? &T : nullptr));
        CK(launch_fam_reduce(w.tiles, nf, (int)P.tiles_last, xs_run, fb, N, P.M_last, P.RL, w.fm, fb,
                             (marg && !fine) ? w.Wf : nullptr, nr, st, perm));
        count_launches(1);
        if (marg) {
            CK(launch_zrange_select(w.Wf, nr, nf, fb, z_per_x, seed, counter0, w.draws, perm, st));
            count_launches(1);
            PassArgs c = b;
            c.src = w.inter;
            c.lo_g = 0;
            CK(launch_zsample(P.npass == 1, fine ? 1 : 0, P.M_last, c, w.draws, z_per_x, w.zs, w.cz, perm, st));
            count_launches(1);
        }
    }
    CK(launch_mc_stats(w.fm, w.cz, n_x, z_per_x, N, marg ? 1 : 0, w.y, w.out, st));
    count_launches(2);
    double h[24];
    CK(cudaMemcpyAsync(h, w.out, 19 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h + 20, w.scal + SCAL_NORM2, sizeof(double), cudaMemcpyDeviceToHost, st));
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    h[21] = 0.0;
    if (marg) CK(cudaMemcpyAsync(h + 21, w.p, sizeof(double), cudaMemcpyDeviceToHost, st));   // p(0) = CDF(0)
    if (xs_dev) CK(cudaMemcpyAsync(xs_dev, w.xs, n_x * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
    if (marg && zs_dev)
        CK(cudaMemcpyAsync(zs_dev, w.zs, (size_t)n_x * z_per_x * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
    if (marg && c_dev)
        CK(cudaMemcpyAsync(c_dev, w.cz, (size_t)n_x * z_per_x * sizeof(float), cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    if (timing) CS(timer_fold(T));
    if (herr & SRE_ERR_TIMEOUT) return fail(SRE_ETIMEOUT, "a bounded device wait of the z sampler expired");
    if (!(h[20] > 0.0)) return fail(SRE_EZERO, "psi has zero norm");

    init_result(out);
    const double dd = (double)d;
    if (!marg) {
        const double nm = (double)(n_x - 1);
        for (int k = 0; k < 3; ++k) {
            const double mean = h[k] / nm;
            const double shat = h[12 + k] + (dd - 1.0) * mean;
            double var = h[6 + k] / nm - mean * mean;
            if (var < 0) var = 0;
            if (k == 0) {
                out->M[0] = shat - N;
                out->S[0] = shat;
                out->err_M[0] = (dd - 1.0) * std::sqrt(var / nm);
            } else {
                const double alpha = k + 1.0;
                out->M[k] = std::log2(shat) / (1.0 - alpha) - N;
                out->S[k] = shat;
                const double r = std::sqrt(var) / (shat / dd);
                out->err_M[k] = r / (std::fabs(1.0 - alpha) * std::log(2.0) * std::sqrt((double)n_x));
                if (k == 1) out->r2 = r;      // sampled Std_{x != 0}(m_x) / E_x[m_x]
            }
            out->M_rb[k] = out->M[k];
            out->err_rb[k] = out->err_M[k];
        }
        out->parseval = -1.0;
    } else {
        // x = 0 stratum (exact) + families 1.. drawn from p(x | x != 0)
        const double n = (double)(n_x - 1);
        const double p0 = h[21];
        for (int which = 0; which < 2; ++which) {
            for (int k = 0; k < 3; ++k) {
                const int idx = k + 3 * which;
                const double mean = h[idx] / n;
                double var = h[6 + idx] / n - mean * mean;
                if (var < 0) var = 0;
                const double S = p0 * h[12 + idx] + (1.0 - p0) * mean;
                const double se = (1.0 - p0) * std::sqrt(var / n);
                double Mv, ev;
                if (k == 0) { Mv = S; ev = se; }
                else {
                    const double alpha = k + 1.0;
                    Mv = std::log2(S) / (1.0 - alpha);
                    ev = se / (S * std::fabs(1.0 - alpha) * std::log(2.0));
                }
                if (which == 0) { out->M[k] = Mv; out->err_M[k] = ev; out->S[k] = S; }
                else { out->M_rb[k] = Mv; out->err_rb[k] = ev; }
            }
        }
        out->parseval = -1.0;
        out->n_samples = n_x * (long long)z_per_x;
    }
    out->n_families = n_x;
    out->n_passes = P.npass;
    return SRE_OK;
}

sre_status pauli_x_marginal(const void *psi, int N, double *p_dev, void *workspace, size_t workspace_bytes,
                            void *stream) {
    CS(check_psi(psi, N, 1, 30));
    if (!p_dev || (((uintptr_t)p_dev) & 7)) return fail(SRE_EINVAL, "p_dev must be a non-NULL 8-byte aligned pointer");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t need = sizeof(double) * ((1ULL << N) + SCAL_N + NORM_BLOCKS) + 4096;
    void *base = nullptr;
    CS(resolve_workspace(workspace, workspace_bytes, need, &base));
    Arena A(base);
    double *scal = A.take<double>(SCAL_N);
    double *part = A.take<double>(NORM_BLOCKS);
    double *mwork = A.take<double>(1ULL << N);
    CK(launch_norm2((const float2 *)psi, N, scal, part, st));
    count_launches(2);
    CS(run_marginal(psi, N, scal, p_dev, mwork, st));
    double nrm = 0;
    CK(cudaMemcpyAsync(&nrm, scal + SCAL_NORM2, sizeof nrm, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!(nrm > 0.0)) return fail(SRE_EZERO, "psi has zero norm");
    return SRE_OK;
}

sre_status stabilizer_nullity(const void *psi, int N, double eps, int *nullity_host, long long *stab_count_host,
                              void *stream) {
    CS(check_psi(psi, N, 1, 26));
    sre_opts o;
    sre_default_opts(&o);
    if (!(eps < 0.5)) return fail(SRE_EINVAL, "eps must lie in (0, 0.5) (or be <= 0: 1e-6)");
    o.eps_null = eps > 0 ? eps : 1e-6;
    sre_result r;
    sre_status s = exact_impl(psi, N, o, nullptr, 0, (cudaStream_t)stream, &r);
    if (nullity_host) *nullity_host = r.nullity;
    if (stab_count_host) *stab_count_host = r.stab_count;
    return s;
}

sre_status sre_family_spectrum(const void *psi, int N, unsigned long long x, const sre_opts *opts, float *c_dev,
                               void *stream) {
    CS(check_psi(psi, N, 1, 30));
    if (!c_dev || (((uintptr_t)c_dev) & 3)) return fail(SRE_EINVAL, "c_dev must be a non-NULL aligned pointer");
    if (x >> N) return fail(SRE_EINVAL, "x has bits above N");
    sre_opts o;
    CS(check_opts(opts, o));
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    CS(plan_for_tuned(N, &o, 32, P));
    void *base = nullptr;
    CS(own_workspace(sizeof(double) * (SCAL_N + NORM_BLOCKS) + P.slot_bytes + 4096, &base));
    Arena A(base);
    double *scal = A.take<double>(SCAL_N);
    double *part = A.take<double>(NORM_BLOCKS);
    void *inter = P.npass > 1 ? (void *)A.take<char>(P.slot_bytes) : nullptr;
    CK(launch_norm2((const float2 *)psi, N, scal, part, st));
    count_launches(2);
    PassArgs a = base_args(P, psi, scal);
    a.precision = prec_code(o);
    a.fam_base = (long long)x;
    a.n_fam = 1;
    a.spec_out = c_dev;
    CS(run_transform(P, a, SRC_PSI_FAMILY, DST_SPECTRUM, inter, st));
    CK(cudaStreamSynchronize(st));
    return SRE_OK;
}

// FP64 spectrum of one family (the arithmetic of the nullity recheck).
sre_status sre_family_spectrum_f64(const void *psi, int N, unsigned long long x, double *c_dev, void *stream) {
    CS(check_psi(psi, N, 1, 28));
    if (!c_dev || (((uintptr_t)c_dev) & 7)) return fail(SRE_EINVAL, "c_dev must be a non-NULL aligned pointer");
    if (x >> N) return fail(SRE_EINVAL, "x has bits above N");
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    CS(plan_for(N, nullptr, 64, P));
    void *base = nullptr;
    CS(own_workspace(sizeof(double) * (SCAL_N + NORM_BLOCKS) + P.slot_bytes + 4096, &base));
    Arena A(base);
    double *scal = A.take<double>(SCAL_N);
    double *part = A.take<double>(NORM_BLOCKS);
    void *inter = P.npass > 1 ? (void *)A.take<char>(P.slot_bytes) : nullptr;
    CK(launch_norm2((const float2 *)psi, N, scal, part, st));
    count_launches(2);
    PassArgs a = base_args(P, psi, scal);
    a.fam_base = (long long)x;
    a.n_fam = 1;
    a.spec_out = c_dev;
    CS(run_transform(P, a, SRC_PSI_FAMILY, DST_SPECTRUM, inter, st));
    CK(cudaStreamSynchronize(st));
    return SRE_OK;
}

sre_status apply_clifford_tdoped_circuit(void *psi, int N, const sre_gate *gates, long long n_gates, void *stream) {
    CS(check_psi(psi, N, 1, 32));
    if (n_gates < 0 || (n_gates > 0 && !gates)) return fail(SRE_EINVAL, "bad gate list");
    for (long long g = 0; g < n_gates; ++g) {
        const sre_gate &G = gates[g];
        if (G.op > SRE_GATE_TDG) return fail(SRE_EINVAL, "gate %lld: unknown op %d", g, G.op);
        if (G.q0 >= N) return fail(SRE_EINVAL, "gate %lld: qubit %d >= N", g, G.q0);
        if (G.op == SRE_GATE_CNOT && (G.q1 >= N || G.q1 == G.q0))
            return fail(SRE_EINVAL, "gate %lld: bad CNOT target %d", g, G.q1);
    }
    std::vector<GateRow> rows((size_t)n_gates);
    for (long long g = 0; g < n_gates; ++g) {
        rows[g].op = gates[g].op;
        rows[g].q0 = gates[g].q0;
        rows[g].q1 = gates[g].op == SRE_GATE_CNOT ? gates[g].q1 : 0;
    }
    return run_gate_list(psi, N, rows, nullptr, (cudaStream_t)stream);
}

sre_status apply_two_qubit_gates(void *psi, int N, const float *mats, const int *pairs, long long n_gates,
                                 void *stream) {
    CS(check_psi(psi, N, 2, 32));
    if (n_gates < 0 || (n_gates > 0 && (!mats || !pairs))) return fail(SRE_EINVAL, "bad gate list");
    std::vector<GateRow> rows((size_t)n_gates);
    for (long long g = 0; g < n_gates; ++g) {
        const int q0 = pairs[2 * g], q1 = pairs[2 * g + 1];
        if (q0 < 0 || q1 < 0 || q0 >= N || q1 >= N || q0 == q1)
            return fail(SRE_EINVAL, "gate %lld: bad qubit pair (%d, %d) for N=%d", g, q0, q1, N);
        rows[g].op = GATE_OP_U2;
        rows[g].q0 = (unsigned char)q0;
        rows[g].q1 = (unsigned char)q1;
    }
    return run_gate_list(psi, N, rows, mats, (cudaStream_t)stream);
}

sre_status sre_mixed_workspace_bytes(int N, int N_A, size_t *bytes) {
    if (N < 1 || N > 30) return fail(SRE_EINVAL, "N=%d outside 1..30", N);
    if (N_A < 1 || N_A > N || N_A > 15) return fail(SRE_EINVAL, "N_A=%d outside 1..min(N, 15)", N_A);
    if (!bytes) return fail(SRE_EINVAL, "bytes is NULL");
    Arena dry(nullptr);
    MixedWS w;
    layout_mixed(dry, N, N_A, w);
    *bytes = dry.off;
    return SRE_OK;
}

sre_status sre_mixed(const void *psi, int N, int N_A, void *workspace, size_t workspace_bytes, void *stream,
                     sre_mixed_result *out) {
    CS(check_psi(psi, N, 1, 30));
    if (N_A < 1 || N_A > N || N_A > 15) return fail(SRE_EINVAL, "N_A=%d outside 1..min(N, 15)", N_A);
    if (!out) return fail(SRE_EINVAL, "out is NULL");
    size_t need = 0;
    CS(sre_mixed_workspace_bytes(N, N_A, &need));
    void *ws = workspace;
    if (!ws) CS(own_workspace(need, &ws));
    else if (workspace_bytes < need) return fail(SRE_EINVAL, "workspace of %zu bytes, %zu needed", workspace_bytes, need);
    return mixed_impl(psi, N, N_A, ws, need, (cudaStream_t)stream, out);
}

unsigned long long sre_kernel_launches(void) { return g_launches.load(); }

unsigned long long sre_device_allocations(void) { return g_allocs.load(); }

// 16 source bytes and the error word of the bounded-wait self-test
__device__ __align__(16) int g_selftest_words[8];

sre_status sre_selftest_queue_wait(void *stream) {
    // one row item whose strided items never run: its dependency wait can
    // only end by its bound
    cudaStream_t st = (cudaStream_t)stream;
    Arena dry(nullptr);
    auto lay = [](Arena &A, BatchBucket *&bk, BatchSeg *&sg, unsigned *&u, unsigned long long *&nx, int *&fl) {
        bk = A.take<BatchBucket>(1);
        sg = A.take<BatchSeg>(1);
        u = A.take<unsigned>(8);
        nx = A.take<unsigned long long>(1);
        fl = A.take<int>(2);
    };
    BatchBucket *bk;
    BatchSeg *sg;
    unsigned *u;
    unsigned long long *nx;
    int *fl;
    lay(dry, bk, sg, u, nx, fl);
    void *base = nullptr;
    CS(own_workspace(dry.off, &base));
    Arena A(base);
    lay(A, bk, sg, u, nx, fl);
    CK(cudaMemsetAsync(base, 0, dry.off, st));
    BatchSeg h;
    memset(&h, 0, sizeof h);
    h.kind = BI_ROW;
    h.aux = 1;
    h.count = 1;
    const unsigned need[2] = {1u, 1u};      // need_str[0] = 1 with no strided item
    CK(cudaMemcpyAsync(sg, &h, sizeof h, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(u, need, sizeof need, cudaMemcpyHostToDevice, st));
    BatchQueue q;
    memset(&q, 0, sizeof q);
    q.segs = sg;
    q.n_segs = 1;
    q.n_items = 1;
    q.buckets = bk;
    q.next = nx;
    q.need_str = u;
    q.need_row = u + 1;
    q.done_str = u + 2;
    q.done_row = u + 3;
    q.ring = PERSIST_RING;
    q.fpc = PERSIST_FPC;
    q.err = fl;
    q.abort_flag = fl + 1;
    CK(launch_batch_persistent(q, true, 1, st));
    count_launches(1);
    int err = 0;
    CK(cudaMemcpyAsync(&err, fl, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err & SRE_ERR_TIMEOUT) return fail(SRE_ETIMEOUT, "queue dependency wait expired (self-test: expected)");
    return SRE_OK;
}

sre_status sre_selftest_bounded_wait(void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    void *base = nullptr;
    CK(cudaGetSymbolAddress(&base, g_selftest_words));
    int *words = reinterpret_cast<int *>(base);
    CK(cudaMemsetAsync(words, 0, sizeof(int) * 8, st));
    CK(launch_wait_selftest(words, words + 4, st));
    count_launches(1);
    int err = 0;
    CK(cudaMemcpyAsync(&err, words + 4, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err & SRE_ERR_TIMEOUT) return fail(SRE_ETIMEOUT, "bounded wait expired (self-test: expected)");
    return SRE_OK;
}

sre_status sre_pass_timing(int enable, double *ms_sum_host, long long *launches_host, double *bytes_host) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    if (ms_sum_host)
        for (int p = 0; p < 4; ++p) ms_sum_host[p] = g_timing_ms[p];
    if (launches_host)
        for (int p = 0; p < 4; ++p) launches_host[p] = g_timing_n[p];
    if (bytes_host)
        for (int p = 0; p < 4; ++p) bytes_host[p] = g_timing_bytes[p];
    if (enable) {
        for (int p = 0; p < 4; ++p) { g_timing_ms[p] = 0; g_timing_n[p] = 0; g_timing_bytes[p] = 0; }
    }
    g_timing_on = enable != 0;
    return SRE_OK;
}

sre_status sre_profile_passes(const void *psi, int N, long long n_x, const sre_opts *opts, void *stream,
                              double *ms_host, double *bytes_host, int *n_passes, long long *fam_per_launch) {
    CS(check_psi(psi, N, 2, 30));
    if (n_x < 1 || !ms_host || !bytes_host || !n_passes || !fam_per_launch)
        return fail(SRE_EINVAL, "bad profile arguments");
    sre_opts o;
    CS(check_opts(opts, o));
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    CS(plan_for_tuned(N, &o, 32, P));
    Arena dry(nullptr);
    McWS w;
    layout_mc(dry, P, SRE_MC_UNIFORM, n_x < 2 ? 2 : n_x, 1, w);
    void *base = nullptr;
    CS(own_workspace(dry.off, &base));
    Arena A(base);
    layout_mc(A, P, SRE_MC_UNIFORM, n_x < 2 ? 2 : n_x, 1, w);
    CK(launch_norm2((const float2 *)psi, N, w.scal, w.npart, st));
    count_launches(2);
    CK(launch_draw_x(nullptr, N, n_x, 0, 12345ULL, 0ULL, w.xs, st));
    count_launches(1);
    PassArgs a = base_args(P, psi, w.scal);
    a.precision = prec_code(o);
    a.xs = w.xs;
    a.tile_out = w.tiles;
    const long long step = P.B < n_x ? P.B : n_x;
    PassTimer T;
    for (long long fb = 0; fb < n_x; fb += step) {
        PassArgs b = a;
        b.fam_base = fb;
        b.n_fam = n_x - fb < step ? n_x - fb : step;
        CS(run_transform(P, b, SRC_PSI_FAMILY, DST_MOMENTS, w.inter, st, &T));
    }
    CK(cudaStreamSynchronize(st));
    double sum[4] = {0, 0, 0, 0};
    int cnt[4] = {0, 0, 0, 0};
    for (size_t i = 0; i < T.pass.size(); ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, T.ev[2 * i], T.ev[2 * i + 1]));
        sum[T.pass[i]] += ms;
        cnt[T.pass[i]] += 1;
    }
    for (cudaEvent_t e : T.ev) cudaEventDestroy(e);
    *n_passes = P.npass;
    *fam_per_launch = step;
    const double d = std::ldexp(1.0, N);
    for (int p = 0; p < P.npass; ++p) {
        ms_host[p] = cnt[p] ? sum[p] / cnt[p] : 0.0;
        // algorithmic bytes per family of pass p: the first pass reads psi
        // (8 B per amplitude, once); every pass but the last writes the
        // packed intermediate (8 B per complex point, d/2 points); every
        // pass but the first reads it.
        double b = 0.0;
        if (p == 0) b += 8.0 * d;
        if (p > 0) b += 4.0 * d;
        if (p < P.npass - 1) b += 4.0 * d;
        bytes_host[p] = b * (double)step;
    }
    return SRE_OK;
}

// Philox4x64-10 blocks for host-side checks of the device generator:
// ctr_key_dev n x (c0,c1,c2,c3,k0,k1), out_dev n x 4 words.
sre_status sre_philox_blocks(const unsigned long long *ctr_key_dev, unsigned long long *out_dev, int n, void *stream) {
    if (n < 0 || (n > 0 && (!ctr_key_dev || !out_dev))) return fail(SRE_EINVAL, "bad philox arguments");
    if (n == 0) return SRE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    CK(launch_philox_test(ctr_key_dev, out_dev, n, st));
    count_launches(1);
    CK(cudaStreamSynchronize(st));
    return SRE_OK;
}

sre_status sre_tc_gemm_selftest(const void *A_bf16_dev, const void *B_bf16_dev, float *D_dev, int M, int N, int K,
                                int swizzle, int *err_dev, void *stream) {
    if (!A_bf16_dev || !B_bf16_dev || !D_dev || !err_dev) return fail(SRE_EINVAL, "tc gemm self-test: NULL pointer");
    if (M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 128 || K % 64)
        return fail(SRE_EINVAL, "tc gemm self-test: M, N must be multiples of 128 and K of 64 (got %d, %d, %d)", M, N, K);
    if (((uintptr_t)A_bf16_dev | (uintptr_t)B_bf16_dev) & 15) return fail(SRE_EINVAL, "tc gemm self-test: operands must be 16-byte aligned");
    if (swizzle != 128 && swizzle != 64 && swizzle != 32)
        return fail(SRE_EINVAL, "tc gemm self-test: swizzle must be 128, 64 or 32");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(err_dev, 0, sizeof(int), st));
    CK(launch_tc05_gemm_selftest(A_bf16_dev, B_bf16_dev, D_dev, M, N, K, swizzle, err_dev, st));
    count_launches(1);
    int h = 0;
    CK(cudaMemcpyAsync(&h, err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h & SRE_ERR_TIMEOUT) return fail(SRE_ETIMEOUT, "tc gemm self-test: a bounded wait ran out");
    return SRE_OK;
}

} // extern "C"
