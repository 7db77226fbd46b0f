// Batched (serving) launches of the bit-layout interval kernel: many realizations of different L
// and R advance by one exchange interval per launch of one persistent-style kernel.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_bits.cuh"

namespace rfim {

// One resident realization ("slot") as the batched kernel sees it.
struct SlotDesc {
  RealView v;
  const float4 *field4;
  ExchArgs xa;      // partials [R] (one slab), arrival counter, J, h
  int32_t L, kind;  // kind: bimodal or float field
  int32_t G, GT;    // replicas per work item, replicas per thread
  int32_t nitems;   // work items of this slot in the queue
  int32_t pad;
};

// One work item: replicas [r0, r0 + gact) of slot `slot`.
struct BatchItem {
  int32_t slot, r0, gact, pad;
};

// Work queue: CTAs take items in order (largest first); the last CTA to leave resets it.
struct BatchQueue {
  unsigned int head;
  unsigned int done_ctas;
  int32_t nitems;
  int32_t pad;
};

constexpr int kBatchThreads = 512;

// Whether a batched instance exists for (L, GT); dynamic shared memory needed for G replicas.
bool batch_supported(int L, int GT);
size_t batch_smem(int L, int G);
int batch_max_gt(int L);
cudaError_t batch_prepare(size_t smem);
cudaError_t batch_occupancy(size_t smem, int *blocks_per_sm);
cudaError_t launch_batch(int grid, size_t smem, const SlotDesc *slots, SlotCtl *ctls, const BatchItem *items,
                         BatchQueue *queue, cudaStream_t st);

}  // namespace rfim
