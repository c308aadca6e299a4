// k_batch.cu -- the exact sweeps of many states of uneven N in one
// persistent launch (Algorithm 1 per state).
//
// The host lays the work out as a queue of items (runs of items described by
// segments, see k_batch.cuh):
//   BI_SINGLE  a single-pass tile (N <= 14): G families of one state, their
//              moments straight into the family sums;
//   BI_STRIDED the strided pass of FPC families of a family batch of a
//              two-pass state (N >= 15), one tile, into the batch's slot of an
//              intermediate ring;
//   BI_ROW     the row pass of RPI families of a batch, each with all its
//              tiles in turn and the fused moments into a tile-partial ring,
//              then the family's sums in tile order.
// The default sweep queues only single-pass items (DEP = false): they are
// independent, and two-pass states keep their own launches. With DEP = true
// the queue holds every family of every state, in dependency order: a batch's
// row items wait until all its strided items are done, and a batch's strided
// items wait until the batch that last used its ring slot is done. Every item
// waits only on items earlier in the queue, which were dequeued by CTAs
// already running, so the launch makes progress whatever the number of
// resident CTAs. Each wait is bounded (about a second of the global timer):
// past the bound the CTA raises SRE_ERR_TIMEOUT and an abort flag, after
// which every CTA drops the rest of the queue.
#include "k_pass_dispatch.cuh"
#include "k_batch.cuh"

namespace sre {

namespace {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long WAIT_NS = 1000000000ull;     // one second

// Wait (thread 0) until *ctr >= need; false on abort or after WAIT_NS.
__device__ bool wait_count(const unsigned *ctr, unsigned need, int *abort_flag, int *err) {
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= need) return true;
        if (*(volatile int *)abort_flag) return false;
        if (global_ns() - t0 > WAIT_NS) {
            atomicOr(err, SRE_ERR_TIMEOUT);
            atomicExch(abort_flag, 1);
            return false;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
}

__device__ __forceinline__ void release_add(unsigned *ctr, unsigned v) {
    __threadfence();
    atomicAdd(ctr, v);
}

// The pass bodies are separate functions so that each is register-allocated
// on its own rather than together with every other instantiation.
template <int M>
__device__ __noinline__ void run_single(const PassArgs &a, long long slot0) {
    fwht_pass_body<typename SingleCfgOf<float, M>::type, SRC_PSI_FAMILY, DST_MOMENTS, 0>(a, slot0, 0);
}

template <int K>
__device__ __noinline__ void run_strided(const PassArgs &a, long long slot0, int fpc, unsigned long long tile) {
    typedef TileCfg<float, 13, 13 - K, 5, 1> Cfg;
#pragma unroll 1
    for (int r = 0; r < fpc; ++r) {
        if (slot0 + r >= a.n_fam) break;
        if (r) __syncthreads();                       // the tile buffer is reused
        fwht_pass_body<Cfg, SRC_PSI_FAMILY, DST_BUF, 0>(a, slot0 + r, tile);
    }
}

__device__ __noinline__ void run_row(const PassArgs &a, long long slot, int tiles) {
#pragma unroll 1
    for (int t = 0; t < tiles; ++t) {
        if (t) __syncthreads();                           // the tile buffer is reused
        fwht_pass_body<TileCfg<float, 13, 0, 5, 1>, SRC_BUF, DST_MOMENTS, 0>(a, slot, (unsigned long long)t);
    }
}

}  // namespace

template <bool DEP>
__global__ void __launch_bounds__(256, 2) batch_persistent_kernel(const BatchQueue q) {
    __shared__ long long s_item;
    __shared__ int s_seg;
    __shared__ __align__(16) PassArgs s_args;            // arguments of the current two-pass item
    __shared__ int s_ok;
    __shared__ int s_have_kind, s_have_batch;           // whose arguments s_args holds (dependency met)
    __shared__ long long s_seg_end;
    const int tid = threadIdx.x;
    // thread 0's next item: taken from the queue while the current item runs,
    // needed only at the top of the next iteration
    unsigned long long next_it = 0;
    if (tid == 0) {
        next_it = atomicAdd(q.next, 1ull);
        s_seg = 0;
        s_seg_end = 0;
        s_have_kind = -1;
        s_have_batch = -1;
    }
#pragma unroll 1
    for (;;) {
        __syncthreads();                                 // the previous item is done with s_item and smem
        if (tid == 0) {
            // the item taken from the queue one item ago (its dequeue ran during
            // the previous item's work)
            long long it = (long long)next_it;
            if (it >= q.n_items) it = -1;
            if constexpr (DEP) {
                if (*(volatile int *)q.abort_flag) it = -1;
            }
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
        const long long l = it - sg.start;
        struct { int kind, bucket, batch, tile; long long slot0; } item;
        item.kind = sg.kind;
        item.bucket = sg.bucket;
        item.batch = sg.batch;
        if (sg.kind == BI_SINGLE) { item.slot0 = l * sg.aux; item.tile = 0; }
        else if (sg.kind == BI_STRIDED) { item.tile = (int)(l / sg.aux); item.slot0 = (l % sg.aux) * q.fpc; }
        else { item.slot0 = l * sg.aux; item.tile = 0; }
        const BatchBucket &bk = q.buckets[item.bucket];
        if (tid == 0) next_it = atomicAdd(q.next, 1ull);
        if (item.kind == BI_SINGLE) {
            switch (bk.M) {
#define C(m) case m: run_single<m>(bk.single, item.slot0); break;
            C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13)
#undef C
            default: break;
            }
            continue;
        }
        if constexpr (!DEP) continue;      // never queued without dependencies
        // two-pass items: the batch's families, intermediate and tile-partial
        // slots. The item's pass arguments are built once in shared memory
        // (a per-thread copy would spill).
        const int kk = item.batch - bk.first_batch;       // batch within the bucket
        const int rs = item.batch % q.ring;               // ring slot (shared by all buckets in turn)
        const long long fb = (long long)kk * bk.B;
        const long long nf = bk.fam_total - fb < bk.B ? bk.fam_total - fb : bk.B;
        if (s_have_kind != item.kind || s_have_batch != item.batch) {
            // (when the CTA's previous two-pass item was of the same pass and
            // batch, its arguments are in place and its dependency is met)
        {
            // the pass's arguments, copied by 8-byte words across the threads
            static_assert(sizeof(PassArgs) % 8 == 0, "PassArgs copies in 8-byte words");
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(
                item.kind == BI_STRIDED ? &bk.strided : &bk.row);
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(&s_args);
            for (int w = tid; w < (int)(sizeof(PassArgs) / 8); w += blockDim.x) dst[w] = src[w];
        }
        __syncthreads();
        if (tid == 0) {
            bool ok;
            if (item.kind == BI_STRIDED) {
                // the ring slot's previous batch (of any bucket) must be done
                ok = item.batch < q.ring ||
                     wait_count(q.done_row + (item.batch - q.ring), q.need_row[item.batch - q.ring], q.abort_flag, q.err);
                s_args.src = s_args.dst = (char *)q.inter + (size_t)rs * q.inter_slot_bytes;
            } else {
                ok = wait_count(q.done_str + item.batch, q.need_str[item.batch], q.abort_flag, q.err);
                s_args.src = (char *)q.inter + (size_t)rs * q.inter_slot_bytes;
                s_args.tile_out = q.tiles + (size_t)rs * q.tiles_slot;
            }
            s_args.fam_base = fb;
            s_args.n_fam = nf;
            s_ok = ok;
            s_have_kind = ok ? item.kind : -1;
            s_have_batch = ok ? item.batch : -1;
        }
        __syncthreads();
        if (!s_ok) continue;
        }
        const PassArgs &a = s_args;
        if (item.kind == BI_STRIDED) {
            switch (bk.K) {
#define C(k) case k: run_strided<k>(a, item.slot0, q.fpc, (unsigned long long)item.tile); break;
            C(1) C(2) C(3) C(4) C(5) C(6)
#undef C
            default: break;
            }
            __syncthreads();
            if (tid == 0) release_add(q.done_str + item.batch, 1u);
            continue;
        }
        // BI_ROW: families slot0 .. slot0 + aux - 1 in turn, every row tile of a
        // family, then its sums in tile order
        const long long fam_end = item.slot0 + sg.aux < nf ? item.slot0 + sg.aux : nf;
#pragma unroll 1
        for (long long f = item.slot0; f < fam_end; ++f) {
            if (f > item.slot0) __syncthreads();          // the tile buffer is reused
            run_row(a, f, bk.tiles_row);
            __syncthreads();
            if (tid < 32) {
                const TilePartial *tp = a.tile_out + (size_t)f * (size_t)bk.tiles_row;
                double m0 = 0, m1 = 0, m2 = 0, m3 = 0, c = 0;
                for (int t = tid; t < bk.tiles_row; t += 32) {
                    m0 += tp[t].m[0]; m1 += tp[t].m[1]; m2 += tp[t].m[2]; m3 += tp[t].m[3];
                    c += (double)tp[t].cand;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    m0 += __shfl_xor_sync(0xffffffffu, m0, o);
                    m1 += __shfl_xor_sync(0xffffffffu, m1, o);
                    m2 += __shfl_xor_sync(0xffffffffu, m2, o);
                    m3 += __shfl_xor_sync(0xffffffffu, m3, o);
                    c += __shfl_xor_sync(0xffffffffu, c, o);
                }
                if (tid == 0) {
                    FamMoments &o = bk.fm[fb + f];
                    o.m[0] = m0; o.m[1] = m1; o.m[2] = m2; o.m[3] = m3;
                    o.cand = (unsigned long long)c;
                }
            }
        }
        if (tid == 0) release_add(q.done_row + item.batch, (unsigned)(fam_end - item.slot0));
    }
}

size_t batch_persistent_smem() {
    // the largest tile of the instantiated configurations plus the reduction scratch
    return sizeof(float2) * (size_t)TileCfg<float, 13, 0, 5, 1>::PSIZE + sizeof(double) * (8 * (256 / 32) + 8);
}

template <bool DEP>
cudaError_t launch_queue(const BatchQueue &q, int grid, cudaStream_t st) {
    static bool attr = false;
    const size_t smem = batch_persistent_smem();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(batch_persistent_kernel<DEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    batch_persistent_kernel<DEP><<<grid, 256, smem, st>>>(q);
    return cudaGetLastError();
}

cudaError_t launch_batch_persistent(const BatchQueue &q, bool dep, int grid, cudaStream_t st) {
    return dep ? launch_queue<true>(q, grid, st) : launch_queue<false>(q, grid, st);
}

}  // namespace sre
