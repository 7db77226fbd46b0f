// Warp-specialised variant of the bit-layout sweep (same arithmetic, same decisions as
// kernels_bits.cuh).  The Philox words of a half-sweep do not depend on the lattice, so 8
// producer warps generate them into shared-memory rings while 16 consumer warps take the
// Metropolis decisions: the multiply-heavy generator and the table / float decision work run in
// different warps and overlap on the SM's pipes instead of alternating inside every warp.
//
// Consumer warp c owns ring c (NS stages of 2 KiB: the four Philox words of one block for its 32
// lanes and GT = 4 replicas); producer warp p fills the rings of consumers 2p and 2p + 1 in the
// order the consumer reads them.  Each stage has a "full" and an "empty" mbarrier (one arrival
// each).  Every wait is bounded: on expiry the warp records an error in the kernel's error word
// and goes on, so the kernel always reaches its barriers and terminates; the host turns the error
// word into RFIM_ETIMEOUT.
#pragma once
#include <cstdint>

#include "kernels_bits.cuh"

namespace rfim {

constexpr int kWsProducerWarps = 8;
constexpr int kWsConsumerWarps = 16;
constexpr int kWsThreads = 32 * (kWsProducerWarps + kWsConsumerWarps);
constexpr int kWsStages = 4;
constexpr int kWsGT = 4;
constexpr int kWsStageBytes = 32 * kWsGT * 16;  // 32 lanes x 4 replicas x uint4
constexpr unsigned kWsSpinLimit = 1u << 20;      // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
      : "memory");
}

// Waits (bounded) for the completion of the phase with the given parity; false on expiry.  After
// the first expiry in the CTA (*abort set) every wait returns false at once, so a broken pipeline
// costs one wait limit, not one per stage.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  const uint32_t a = smem_addr(bar);
  for (unsigned it = 0; it < kWsSpinLimit; ++it) {
    if (*abort) return false;
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  *abort = 1;
  return false;
}

// Same contract as bits_interval (GT = 4, kWsThreads threads).  `err` collects expired waits.
template <int L, int S, bool BIM>
__device__ __forceinline__ void ws_interval(const RealView &v, int G, int r0, int gact, int rank, uint32_t sweep0,
                                            int nsw, const float4 *__restrict__ field4, unsigned int *err) {
  using Gm = BitsGeom<L>;
  constexpr int P = Gm::P, W = Gm::W, PZ = L / S, WC = PZ * P;
  constexpr int64_t WPAD = (W + 31) / 32 * 32;
  constexpr int kItemsPerRound = 32 * kWsConsumerWarps;
  constexpr int kRounds = (WC + kItemsPerRound - 1) / kItemsPerRound;
  constexpr int GT = kWsGT;
  extern __shared__ __align__(16) uint32_t sm[];
  const int up_rank = (rank + 1) % S, dn_rank = (rank + S - 1) % S;
  const int z0 = rank * PZ;
  uint32_t *sp = sm;                                        // [G][2][WC]
  uint32_t *tab = sm + (size_t)G * 2 * WC;                  // G decision-table slots
  uint4 *ring = reinterpret_cast<uint4 *>(tab + tab_bytes(G) / 4);  // [16][NS][GT*32] uint4
  uint64_t *bars = reinterpret_cast<uint64_t *>(ring + (size_t)kWsConsumerWarps * kWsStages * GT * 32);
  // bars: full[16][NS], empty[16][NS]
  const int nt = blockDim.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int t = tid; t < gact * 2 * WC; t += nt) {
    const int g = t / (2 * WC), rem = t % (2 * WC), c = rem / WC, wl = rem % WC;
    sp[t] = v.bits[((int64_t)(r0 + g) * 2 + c) * W + (int64_t)z0 * P + wl];
  }
  const uint32_t slot0 = tab_slot0(tab);
  tab_fill<BIM>(v, tab, slot0, gact, [&](int g) { return r0 + g; });
  __shared__ int ws_abort;
  if (tid == 0) ws_abort = 0;
  if (tid < 2 * kWsConsumerWarps * kWsStages) mbar_init(bars + tid, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  sync_slabs<S>();

  const bool producer = warp < kWsProducerWarps;
  uint32_t use[2] = {0u, 0u};  // stages used so far on this warp's ring(s)
  bool expired = false;
  for (int s = 0; s < nsw; ++s) {
    const uint32_t sweep = sweep0 + (uint32_t)s;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const uint32_t tag = tag_word(kTagMetro, v.stage, (uint32_t)c);
      if (producer) {
        // two consumer rings per producer warp, filled round by round, block by block
#pragma unroll 1
        for (int rd = 0; rd < kRounds; ++rd) {
#pragma unroll 1
          for (int jj = 0; jj < 8; ++jj) {
            const int j = 7 - jj;
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
              const int cw = 2 * warp + h;
              const int item = (rd * kWsConsumerWarps + cw) * 32 + lane;
              const int wl = min(item, WC - 1);
              const int64_t wq = (int64_t)(z0 + wl / P) * P + wl % P;
              const uint32_t u = use[h]++;
              const int st = (int)(u % kWsStages);
              if (!mbar_wait(bars + kWsConsumerWarps * kWsStages + cw * kWsStages + st, ((u / kWsStages) & 1u) ^ 1u,
                             &ws_abort))
                expired = true;
              uint4 *slot = ring + ((size_t)cw * kWsStages + st) * GT * 32;
#pragma unroll
              for (int gg = 0; gg < GT; ++gg) {
                const int g = min(gg, gact - 1);
                const Words4 w = philox10(v.seed, v.realization, (uint32_t)(8 * wq + j), (uint32_t)(r0 + g), sweep, tag);
                slot[gg * 32 + lane] = make_uint4(w.w[0], w.w[1], w.w[2], w.w[3]);
              }
              __syncwarp();
              if (lane == 0) mbar_arrive(bars + cw * kWsStages + st);
            }
          }
        }
      } else {
        const int cw = warp - kWsProducerWarps;
#pragma unroll 1
        for (int rd = 0; rd < kRounds; ++rd) {
          const int item = (rd * kWsConsumerWarps + cw) * 32 + lane;
          const bool live = item < WC;
          const int wl = min(item, WC - 1);
          const int zl = wl / P, iw = wl % P;
          const int z = z0 + zl;
          const int64_t wq = (int64_t)z * P + iw;
          const float4 *f4w = field4 + field4_index(c, wq, 0, WPAD);  // block j at f4w + 32 j
          const uint32_t p0 = parity0_mask<L>(c, z, iw);
          PairSlices ps[GT];
          uint32_t sf[GT], flip[GT], fk[GT][4];
          const uint32_t fb = BIM ? v.hbits[(int64_t)c * W + wq] : 0u;
#pragma unroll
          for (int gg = 0; gg < GT; ++gg) {
            const int g = min(gg, gact - 1);
            uint32_t nb[6], c0, c1, c2;
            neighbour_words<L, S>(sp + ((size_t)g * 2 + (c ^ 1)) * WC, zl, iw, p0, up_rank, dn_rank, nb);
            count6(nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], c0, c1, c2);
            sf[gg] = sp[((size_t)g * 2 + c) * WC + wl];
            ps[gg] = make_pairs(c0, c1, c2, sf[gg], fb);
            flip[gg] = 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) fk[gg][k] = 0u;
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = 7 - jj;
            float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!BIM) q4 = __ldg(f4w + 32 * j);
            const uint32_t u = use[0]++;
            const int st = (int)(u % kWsStages);
            if (!mbar_wait(bars + cw * kWsStages + st, (u / kWsStages) & 1u, &ws_abort)) expired = true;
            const uint4 *slot = ring + ((size_t)cw * kWsStages + st) * GT * 32;
            uint4 wr[GT];
#pragma unroll
            for (int gg = 0; gg < GT; ++gg) wr[gg] = slot[gg * 32 + lane];
            __syncwarp();
            if (lane == 0) mbar_arrive(bars + kWsConsumerWarps * kWsStages + cw * kWsStages + st);
#pragma unroll
            for (int gg = 0; gg < GT; ++gg) {
              const int g = min(gg, gact - 1);
              const Words4 ww = {{wr[gg].x, wr[gg].y, wr[gg].z, wr[gg].w}};
              decide_block<BIM>(ww, ps[gg], j, slot0 + (uint32_t)g * kTabSlot, q4, flip[gg], fk[gg]);
            }
          }
          if (live) {
#pragma unroll
            for (int gg = 0; gg < GT; ++gg) {
              if (gg >= gact) continue;
              if (!BIM) flip[gg] = fk[gg][0] | (fk[gg][1] << 8) | (fk[gg][2] << 16) | (fk[gg][3] << 24);
              sp[((size_t)gg * 2 + c) * WC + wl] = sf[gg] ^ flip[gg];
            }
          }
        }
      }
      sync_slabs<S>();
    }
  }
  if (expired) atomicOr(err, 1u);

  for (int t = tid; t < gact * 2 * WC; t += nt) {
    const int g = t / (2 * WC), rem = t % (2 * WC), c = rem / WC, wl = rem % WC;
    v.bits[((int64_t)(r0 + g) * 2 + c) * W + (int64_t)z0 * P + wl] = sp[t];
  }
}

template <int L, int S, bool BIM>
__global__ void __launch_bounds__(kWsThreads, 1) k_sweeps_ws(RealView v, int32_t G, uint32_t sweep0, int32_t nsw,
                                                             const float4 *__restrict__ field4, ExchArgs xa) {
  const int rank = S > 1 ? (int)cluster_rank() : 0;
  const int r0 = (int)(blockIdx.x / S) * G;
  const int gact = min(G, v.R - r0);
  xa.expected = gridDim.x;
  ws_interval<L, S, BIM>(v, G, r0, gact, rank, sweep0, nsw, field4, xa.err);
  if (xa.enabled) interval_tail<L, S, BIM>(v, G, r0, gact, rank, nsw, field4, xa);
}

// Dynamic shared memory of the warp-specialised kernel for L / S and G replicas.
__host__ __device__ constexpr size_t ws_smem(int L, int S, int G) {
  return (size_t)G * 2 * ((size_t)(L / S) * (L * L / 64)) * 4 + tab_bytes(G) +
         (size_t)kWsConsumerWarps * kWsStages * kWsStageBytes + (size_t)2 * kWsConsumerWarps * kWsStages * 8;
}

}  // namespace rfim
