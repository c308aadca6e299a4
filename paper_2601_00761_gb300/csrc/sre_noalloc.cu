// sre_noalloc.cu -- the exact sweep on a fixed device scratch that the library
// reserves statically, for callers that must not allocate device memory.
//
// The scratch is a file-scope __device__ array: every GPU that loads the
// library holds SRE_NOALLOC_SCRATCH_BYTES for it until the process exits. In
// host code its name stands for a host-side shadow, not a device address, so
// the device address is looked up with cudaGetSymbolAddress once per device
// (on the first call made while that device is current) and cached.
#include <cstdio>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "sre.h"

namespace sre {
void set_error_message(const char *msg);   // sre_api.cu
}

static __device__ __align__(256) unsigned char g_noalloc_scratch[SRE_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
std::vector<void *> g_noalloc_ptr;   // device address of the scratch, per device
}

extern "C" sre_status sre_exact_noalloc(const void *psi_c64_dev, int N, const sre_opts *opts, void *stream,
                                        sre_result *out) {
    char msg[256];
    if (N < 1 || N > SRE_NOALLOC_MAX_N) {
        snprintf(msg, sizeof msg, "sre_exact_noalloc: N=%d outside 1..%d (the fixed scratch holds %u bytes)", N,
                 SRE_NOALLOC_MAX_N, (unsigned)SRE_NOALLOC_SCRATCH_BYTES);
        sre::set_error_message(msg);
        return SRE_EINVAL;
    }
    size_t need = 0;
    sre_status st = sre_workspace_bytes(N, -1, 0, 0, opts, &need);
    if (st != SRE_OK) return st;
    if (need > SRE_NOALLOC_SCRATCH_BYTES) {
        snprintf(msg, sizeof msg, "sre_exact_noalloc: N=%d needs %zu bytes of scratch, the fixed scratch holds %u", N,
                 need, (unsigned)SRE_NOALLOC_SCRATCH_BYTES);
        sre::set_error_message(msg);
        return SRE_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "sre_exact_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
        sre::set_error_message(msg);
        return SRE_ECUDA;
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if ((int)g_noalloc_ptr.size() <= dev) g_noalloc_ptr.resize(dev + 1, nullptr);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                snprintf(msg, sizeof msg, "sre_exact_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                sre::set_error_message(msg);
                return SRE_ECUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    // sre_exact on a caller workspace allocates nothing; it clears the parts
    // of the workspace that must start at zero before use.
    return sre_exact(psi_c64_dev, N, opts, scratch, SRE_NOALLOC_SCRATCH_BYTES, stream, out);
}
