// Persistent-style batched kernel: a fixed grid of CTAs pulls work items (replica groups of
// resident realizations) from a device queue and runs one exchange interval per item with the
// same device function as the single-realization launch (kernels_bits.cuh, one slab per
// replica).  The last item of each realization takes its exchange step and advances the
// realization's counters on the device, so a captured graph of such launches needs no host
// input between launches.  Realizations never interact: each one's arithmetic, partial sums and
// decisions are those of a solo run with the same replica grouping.
#include "batch.h"

namespace rfim {

namespace {

template <int L, int GT>
__device__ __forceinline__ void run_item(const SlotDesc &sd, const BatchItem &bi, SlotCtl *ctl) {
  ExchArgs xa = sd.xa;
  xa.enabled = 1;
  xa.j = ctl->j;
  xa.measure_from = ctl->measure_from;
  xa.expected = (unsigned)sd.nitems;
  xa.ctl = ctl;
  const uint32_t sweep0 = ctl->sweep0;
  const int nsw = ctl->nsw;
  if (sd.kind == kBimodal)
    bits_interval<L, 1, GT, true, true>(sd.v, sd.G, bi.r0, bi.gact, 0, sweep0, nsw, sd.field4, xa);
  else
    bits_interval<L, 1, GT, false, true>(sd.v, sd.G, bi.r0, bi.gact, 0, sweep0, nsw, sd.field4, xa);
}

__global__ void __launch_bounds__(kBatchThreads) k_batch_bits(const SlotDesc *__restrict__ slots, SlotCtl *ctls,
                                                              const BatchItem *__restrict__ items, BatchQueue *q) {
  __shared__ int s_item;
  const int nitems = q->nitems;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&q->head, 1u);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const BatchItem bi = items[it];
    SlotCtl *ctl = ctls + bi.slot;
    if (ctl->intervals_left <= 0) continue;  // finished realization: its items idle until retired
    const SlotDesc &sd = slots[bi.slot];
    switch (sd.L * 4 + sd.GT) {
      case 64 * 4 + 1: run_item<64, 1>(sd, bi, ctl); break;
      case 64 * 4 + 2: run_item<64, 2>(sd, bi, ctl); break;
      case 32 * 4 + 1: run_item<32, 1>(sd, bi, ctl); break;
      case 32 * 4 + 2: run_item<32, 2>(sd, bi, ctl); break;
      case 16 * 4 + 1: run_item<16, 1>(sd, bi, ctl); break;
      case 8 * 4 + 1: run_item<8, 1>(sd, bi, ctl); break;
      default: break;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&q->done_ctas, 1u);
    if (prev == gridDim.x - 1) {
      q->head = 0u;
      q->done_ctas = 0u;
      __threadfence();
    }
  }
}

}  // namespace

bool batch_supported(int L, int GT) {
  switch (L) {
    case 64: return GT == 1 || GT == 2;
    case 32: return GT == 1 || GT == 2;
    case 16: return GT == 1;
    case 8: return GT == 1;
    default: return false;
  }
}

int batch_max_gt(int L) { return (L == 64 || L == 32) ? 2 : 1; }

size_t batch_smem(int L, int G) { return (size_t)G * 2 * ((size_t)L * L * L / 64) * 4 + tab_bytes(G); }

cudaError_t batch_prepare(size_t smem) {
  return raise_smem_limit((const void *)k_batch_bits, smem);
}

cudaError_t batch_occupancy(size_t smem, int *blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_bits, kBatchThreads, smem);
}

cudaError_t launch_batch(int grid, size_t smem, const SlotDesc *slots, SlotCtl *ctls, const BatchItem *items,
                         BatchQueue *queue, cudaStream_t st) {
  k_batch_bits<<<grid, kBatchThreads, smem, st>>>(slots, ctls, items, queue);
  return cudaGetLastError();
}

}  // namespace rfim
