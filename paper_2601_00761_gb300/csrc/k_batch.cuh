// k_batch.cuh -- work items and queue of the persistent batched sweep (k_batch.cu).
#pragma once

#include "sre_internal.cuh"

namespace sre {

// A run of work items of one bucket: item i of the launch belongs to the
// segment with start <= i < start + count, and covers the families
// (i - start) * per_cta ... + per_cta - 1 of the bucket (one per tile group
// of the CTA; a family is one single-pass tile).
struct BatchSeg {
    int bucket;         // index into BatchQueue::buckets
    int per_cta;        // families per CTA (the single-pass tile's groups)
    long long start, count;
};

// One bucket (states of one N <= 14) as the persistent kernel sees it.
struct BatchBucket {
    PassArgs single;    // fam_base 0, n_fam all families, psi_list / s_list per state, fam_out = fm
    int M;              // tile bits (N - 1)
};

struct BatchQueue {
    const BatchSeg *segs;
    int n_segs;
    long long n_items;
    const BatchBucket *buckets;
    unsigned long long *next;    // queue head (zeroed before the launch)
};

size_t batch_persistent_smem();
cudaError_t launch_batch_persistent(const BatchQueue &q, int grid, cudaStream_t st);

}  // namespace sre
