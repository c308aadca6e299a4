// k_batch.cuh -- work items and queue of the persistent batched sweep (k_batch.cu).
#pragma once

#include "sre_internal.cuh"

namespace sre {

enum BatchItemKind { BI_SINGLE = 0, BI_STRIDED = 1, BI_ROW = 2 };

// A run of work items of one kind, bucket and batch; item i of the launch
// belongs to the segment with start <= i < start + count. Decoding the local
// index l = i - start:
//   BI_SINGLE:  slot0 = l * aux (aux = families per CTA)
//   BI_STRIDED: tile = l / aux, slot0 = (l % aux) * fpc (aux = family groups
//               of the batch; tiles outer, so the CTAs in flight share a tile)
//   BI_ROW:     slot0 = l * aux (aux = families per CTA, all their row tiles)
struct BatchSeg {
    int kind;           // BatchItemKind
    int bucket;         // index into BatchQueue::buckets
    int batch;          // two-pass: global family-batch id (dependency counters, ring slot)
    int aux;
    long long start, count;
};

// One bucket (states of one N) as the persistent kernel sees it.
struct BatchBucket {
    PassArgs single;    // single-pass sweep (N <= 14): fam_base 0, n_fam all families, fam_out = fm
    PassArgs strided;   // two-pass: first pass (SRC_PSI_FAMILY -> DST_BUF), src/dst set per batch
    PassArgs row;       // two-pass: last pass (SRC_BUF -> DST_MOMENTS), src/tile_out set per batch
    FamMoments *fm;     // family sums of the bucket, index (state << N) | x
    long long fam_total;  // families of the bucket
    long long B;        // families per batch (two-pass)
    int M;              // single-pass tile bits (N - 1)
    int K;              // two-pass: rows of the strided pass (N - 14)
    int tiles_row;      // two-pass: tiles per family of the row pass
    int first_batch;    // global id of the bucket's first batch
};

// The queue of one launch. Without dependencies (single-pass items only)
// the fields from done_str on are unused.
struct BatchQueue {
    const BatchSeg *segs;
    int n_segs;
    long long n_items;
    const BatchBucket *buckets;
    unsigned long long *next;    // queue head (zeroed before the launch)
    unsigned *done_str, *done_row;   // per global batch: strided / row items done (zeroed)
    const unsigned *need_str, *need_row;   // per global batch: item counts
    void *inter;                 // intermediate ring: `ring` slots of inter_slot_bytes
    size_t inter_slot_bytes;
    TilePartial *tiles;          // tile-partial ring: `ring` slots of tiles_slot partials
    size_t tiles_slot;
    int ring;
    int fpc;                     // families per strided item
    int *err;                    // device error word (SRE_ERR_TIMEOUT)
    int *abort_flag;             // set on a timed-out wait (zeroed)
};

size_t batch_persistent_smem();
// dep: the queue holds two-pass items (strided and row items with their
// dependency waits); otherwise only single-pass items.
cudaError_t launch_batch_persistent(const BatchQueue &q, bool dep, int grid, cudaStream_t st);

}  // namespace sre
