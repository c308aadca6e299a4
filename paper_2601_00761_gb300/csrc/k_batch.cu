// k_batch.cu -- the exact sweeps of many small states of uneven N in one
// persistent launch (Algorithm 1 per state, every family x of every state
// whose family transform fits one CTA's tile: N <= 14).
//
// The host lays the families out as a queue of items, bucket by bucket
// (segments of k_batch.cuh); an item is one CTA's single-pass tile: G
// families of one state (G = 256 / 2^(N-6) for N <= 13, 1 for N = 14), their
// moments fused into the tile and written straight into the family sums.
// Persistent CTAs (two per SM) take items from one device counter. The items
// are independent, so nothing waits; each CTA takes its next item while the
// current one runs.
#include "k_pass_dispatch.cuh"
#include "k_batch.cuh"

namespace sre {

namespace {

// The single-pass bodies are separate functions so that each is
// register-allocated on its own rather than together with every other size.
template <int M>
__device__ __noinline__ void run_single(const PassArgs &a, long long slot0) {
    fwht_pass_body<typename SingleCfgOf<float, M>::type, SRC_PSI_FAMILY, DST_MOMENTS, 0>(a, slot0, 0);
}

}  // namespace

__global__ void __launch_bounds__(256, 2) batch_persistent_kernel(const BatchQueue q) {
    __shared__ long long s_item, s_seg_end;
    __shared__ int s_seg;
    const int tid = threadIdx.x;
    // thread 0's next item: taken from the queue while the current item runs,
    // needed only at the top of the next iteration
    unsigned long long next_it = 0;
    if (tid == 0) {
        next_it = atomicAdd(q.next, 1ull);
        s_seg = 0;
        s_seg_end = 0;
    }
#pragma unroll 1
    for (;;) {
        __syncthreads();                                 // the previous item is done with s_item and smem
        if (tid == 0) {
            long long it = (long long)next_it;
            if (it >= q.n_items) it = -1;
            s_item = it;
            // the item's segment: the last with start <= it. A CTA's items come
            // in increasing order, so the search starts at its previous segment
            // (whose end is kept in shared memory) and almost always stops there.
            if (it >= 0 && it >= s_seg_end) {
                int g = s_seg;
                while (g + 1 < q.n_segs && q.segs[g + 1].start <= it) ++g;
                s_seg = g;
                s_seg_end = g + 1 < q.n_segs ? q.segs[g + 1].start : q.n_items;
            }
        }
        __syncthreads();
        const long long it = s_item;
        if (it < 0) return;
        const BatchSeg sg = q.segs[s_seg];
        const BatchBucket &bk = q.buckets[sg.bucket];
        const long long slot0 = (it - sg.start) * sg.per_cta;
        if (tid == 0) next_it = atomicAdd(q.next, 1ull);
        switch (bk.M) {
#define C(m) case m: run_single<m>(bk.single, slot0); break;
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13)
#undef C
        default: break;
        }
    }
}

size_t batch_persistent_smem() {
    // the largest single-pass tile (2^13 points, or G groups of smaller
    // tiles) plus the reduction scratch
    return sizeof(float2) * (size_t)TileCfg<float, 13, 0, 5, 1>::PSIZE + sizeof(double) * (8 * (256 / 32) + 8);
}

cudaError_t launch_batch_persistent(const BatchQueue &q, int grid, cudaStream_t st) {
    static bool attr = false;
    const size_t smem = batch_persistent_smem();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(batch_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    batch_persistent_kernel<<<grid, 256, smem, st>>>(q);
    return cudaGetLastError();
}

}  // namespace sre
