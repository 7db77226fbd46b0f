// Bit-layout (multi-spin coded) checkerboard sweep kernel, resident in shared memory.
//
// One cluster of S CTAs holds G replicas of a realization; CTA `rank` holds the z planes
// [rank L/S, (rank + 1) L/S) of both colours of all G replicas in shared memory for the whole
// launch and runs n sweeps (colour 0 half-sweep, colour 1 half-sweep; Eq. 3) before writing the
// lattices back.  Halo planes z0 - 1 and z0 + L/S come from the neighbouring CTAs of the cluster
// through distributed shared memory; a cluster barrier separates half-sweeps (S = 1: the CTA
// barrier).  A thread updates one 32-site word for GT replicas: neighbour counts by bit-sliced
// adders, then per Philox block (4 sites) one table lookup and one compare per site; the float
// field of those 4 sites is loaded once for all GT replicas.
#pragma once
#include <cstdint>

#include "bits_layout.cuh"
#include "decide.cuh"
#include "internal.h"
#include "philox.cuh"

namespace rfim {

__host__ __device__ __forceinline__ int64_t field4_index(int c, int64_t wq, int j, int64_t wpad) {
  return ((int64_t)c * wpad + (wq & ~31LL)) * 8 + (int64_t)j * 32 + (wq & 31);
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t dsmem_load(const uint32_t *local, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
  uint32_t ra, val;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(val) : "r"(ra) : "memory");
  return val;
}

template <int S>
__device__ __forceinline__ void sync_slabs() {
  if (S == 1) {
    __syncthreads();
  } else {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
}

// bit b of every byte of the result = bit j of the same byte of x (b, j fold to constants
// once the chunk loop is unrolled)
__device__ __forceinline__ uint32_t spread(uint32_t x, int b, int j) {
  const uint32_t s = b >= j ? (x << (b - j)) : (x >> (j - b));
  return s & (0x01010101u << b);
}

template <int L, int S, int GT, bool BIM>
__global__ void __launch_bounds__(512) k_sweeps_bits(RealView v, int32_t G, uint32_t sweep0, int32_t nsw,
                                                     const float4 *__restrict__ field4) {
  using Gm = BitsGeom<L>;
  constexpr int P = Gm::P, W = Gm::W, PZ = L / S, WC = PZ * P;
  constexpr int64_t WPAD = (W + 31) / 32 * 32;
  extern __shared__ __align__(16) uint32_t sm[];
  const int rank = S > 1 ? (int)cluster_rank() : 0;
  const int up_rank = (rank + 1) % S, dn_rank = (rank + S - 1) % S;
  const int r0 = (int)(blockIdx.x / S) * G;
  const int gact = min(G, v.R - r0);
  const int z0 = rank * PZ;
  uint32_t *sp = sm;  // [G][2][WC]
  uint32_t *tab = sm + (size_t)G * 2 * WC;  // BIM: [G][32] uint32; else [G][16] float2
  const int nt = blockDim.x, tid = threadIdx.x;

  for (int t = tid; t < gact * 2 * WC; t += nt) {
    const int g = t / (2 * WC), rem = t % (2 * WC), c = rem / WC, wl = rem % WC;
    sp[t] = v.bits[((int64_t)(r0 + g) * 2 + c) * W + (int64_t)z0 * P + wl];
  }
  if (BIM) {
    for (int t = tid; t < gact * 32; t += nt) {
      const int g = t >> 5;
      tab[t] = v.thr[(int64_t)v.r2t[r0 + g] * 32 + (t & 31)];
    }
  } else {
    float2 *gt = reinterpret_cast<float2 *>(tab);
    for (int t = tid; t < gact * 16; t += nt) {
      const int g = t >> 4, i = t & 15;
      const float b = v.b2[v.r2t[r0 + g]];
      gt[t] = make_float2(v.gjn[i & 7], (i >> 3) ? b : -b);
    }
  }
  sync_slabs<S>();

  const int ngroups = (gact + GT - 1) / GT;
  const int items = WC * ngroups;
  for (int s = 0; s < nsw; ++s) {
    const uint32_t sweep = sweep0 + (uint32_t)s;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const uint32_t tag = tag_word(kTagMetro, v.stage, (uint32_t)c);
#pragma unroll 1
      for (int item = tid; item < items; item += nt) {
        const int wl = item % WC, grp = item / WC;
        const int zl = wl / P, iw = wl % P;
        const int z = z0 + zl;
        const int64_t wq = (int64_t)z * P + iw;
        const uint32_t p0 = parity0_mask<L>(c, z, iw);
        uint32_t c0[GT], c1[GT], c2[GT], sf[GT], flip[GT];
#pragma unroll
        for (int gg = 0; gg < GT; ++gg) {
          const int g = min(grp * GT + gg, gact - 1);
          const uint32_t *O = sp + ((size_t)g * 2 + (c ^ 1)) * WC;
          const uint32_t same = O[zl * P + iw];
          const uint32_t next = O[zl * P + (iw + 1) % P];
          const uint32_t prev = O[zl * P + (iw + P - 1) % P];
          uint32_t A, B, C, D;
          nb_xy<L>(same, next, prev, p0, A, B, C, D);
          uint32_t E, F;
          if (zl + 1 < PZ)
            E = O[(zl + 1) * P + iw];
          else
            E = S == 1 ? O[iw] : dsmem_load(O + iw, up_rank);
          if (zl > 0)
            F = O[(zl - 1) * P + iw];
          else
            F = S == 1 ? O[(PZ - 1) * P + iw] : dsmem_load(O + (PZ - 1) * P + iw, dn_rank);
          count6(A, B, C, D, E, F, c0[gg], c1[gg], c2[gg]);
          sf[gg] = sp[((size_t)g * 2 + c) * WC + wl];
          flip[gg] = 0u;
        }
        uint32_t fb = 0;
        if (BIM) fb = v.hbits[(int64_t)c * W + wq];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float4 hh4 = make_float4(0.f, 0.f, 0.f, 0.f);
          if (!BIM) hh4 = __ldg(field4 + field4_index(c, wq, j, WPAD));
#pragma unroll
          for (int gg = 0; gg < GT; ++gg) {
            const int g = grp * GT + gg;
            if (GT > 1 && g >= gact) continue;
            const Words4 w = philox10(v.seed, v.realization, (uint32_t)(8 * wq + j), (uint32_t)(r0 + g), sweep, tag);
            uint32_t acc;
            if (BIM) {
              acc = spread(c0[gg], 2, j) | spread(c1[gg], 3, j) | spread(c2[gg], 4, j) | spread(sf[gg], 5, j) |
                    spread(fb, 6, j);
            } else {
              acc = spread(c0[gg], 3, j) | spread(c1[gg], 4, j) | spread(c2[gg], 5, j) | spread(sf[gg], 6, j);
            }
            const char *tb = reinterpret_cast<const char *>(tab) + g * 128;
            const float hk[4] = {hh4.x, hh4.y, hh4.z, hh4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t off = (acc >> (8 * k)) & 0xFFu;
              bool a;
              if (BIM) {
                a = accept_table(w.w[k], *reinterpret_cast<const uint32_t *>(tb + off));
              } else {
                const float2 e = *reinterpret_cast<const float2 *>(tb + off);
                a = accept_float(w.w[k], e.x, hk[k], e.y);
              }
              flip[gg] |= (uint32_t)a << (8 * k + j);
            }
          }
        }
#pragma unroll
        for (int gg = 0; gg < GT; ++gg) {
          const int g = grp * GT + gg;
          if (GT > 1 && g >= gact) continue;
          sp[((size_t)g * 2 + c) * WC + wl] = sf[gg] ^ flip[gg];
        }
      }
      sync_slabs<S>();
    }
  }

  for (int t = tid; t < gact * 2 * WC; t += nt) {
    const int g = t / (2 * WC), rem = t % (2 * WC), c = rem / WC, wl = rem % WC;
    v.bits[((int64_t)(r0 + g) * 2 + c) * W + (int64_t)z0 * P + wl] = sp[t];
  }
}

}  // namespace rfim
