// Multi-hit double 3D checkerboard sweeps (Sec. 3.2; the multi-hit runs of Sec. 6) on the bit
// layout.  The lattice is cut into tiles of T^3 sites with coarse colour (x/T + y/T + z/T) mod 2.
// One sweep visits the tiles of coarse colour 0, then those of colour 1; a visit makes mh local
// passes, each a black-white pass (fine colour 0, then 1) over the visited tiles while the
// neighbouring tiles stay frozen.  Pass h of sweep s draws the Philox words of counter
// (q >> 2, r, s mh + h, c3(METRO, stage, fine colour)).
//
// The whole slab already sits in shared memory, so a tile visit needs no load of its own: a pass
// is a masked half-sweep.  With T a multiple of 8, the four sites of a Philox block (x in
// [8 j', 8 j' + 8) of one row) lie in one tile, so a pass skips whole blocks.  Words are handed
// to threads grouped by the parity of (y/T + z/T), so the 32 words of a warp skip the same
// blocks and the skip is a uniform branch.
#pragma once
#include <cstdint>

#include "kernels_bits.cuh"
#include "sweep_bits.h"

namespace rfim {

template <int L, int S, int GT, bool BIM>
__device__ __forceinline__ void bits_interval_mh(const RealView &v, int G, int r0, int gact, int rank, uint32_t sweep0,
                                                 int nsw, const float4 *__restrict__ field4, const ExchArgs &xa,
                                                 const MultiHit &mh) {
  using Gm = BitsGeom<L>;
  constexpr int P = Gm::P, W = Gm::W, PZ = L / S, WC = PZ * P;
  constexpr int RW = 64 / L;  // rows of one colour held by a word
  constexpr int64_t WPAD = (W + 31) / 32 * 32;
  static_assert(L >= 16 && WC % 64 == 0, "a warp's words must share one parity class");
  extern __shared__ __align__(16) uint32_t sm[];
  const int up_rank = (rank + 1) % S, dn_rank = (rank + S - 1) % S;
  const int z0 = rank * PZ;
  __syncthreads();
  uint32_t *sp = sm;
  uint32_t *tab = sm + (size_t)G * 2 * WC;
  const uint32_t slot0 = tab_slot0(tab);
  const int nt = blockDim.x, tid = threadIdx.x;

  for (int t = tid; t < gact * 2 * WC; t += nt) {
    const int g = t / (2 * WC), rem = t % (2 * WC), c = rem / WC, wl = rem % WC;
    sp[t] = v.bits[((int64_t)(r0 + g) * 2 + c) * W + (int64_t)z0 * P + wl];
  }
  tab_fill<BIM>(v, tab, slot0, gact, [&](int g) { return r0 + g; });
  sync_slabs<S>();

  const int ngroups = (gact + GT - 1) / GT;
  const int items = WC * ngroups;
  // tiles and bands are powers of two: words of one tile band (T rows) in a plane = T / RW
  constexpr int RW_LOG2 = RW == 1 ? 0 : RW == 2 ? 1 : 2;
  const int t_log2 = mh.tile_log2, w_log2 = t_log2 - RW_LOG2, wmask = (1 << w_log2) - 1;
  for (int s = 0; s < nsw; ++s) {
    const uint32_t sweep = sweep0 + (uint32_t)s;
#pragma unroll 1
    for (int coarse = 0; coarse < 2; ++coarse) {
#pragma unroll 1
      for (int hit = 0; hit < mh.mh; ++hit) {
        const uint32_t c2 = sweep * (uint32_t)mh.mh + (uint32_t)hit;
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
          const uint32_t tag = tag_word(kTagMetro, v.stage, (uint32_t)c);
#pragma unroll 1
          for (int item = tid; item < items; item += nt) {
            // item -> (replica group, parity class of y/T + z/T, word): each class holds WC / 2
            // words of the slab, P / 2 per plane, in bands of T / RW words of alternate tile rows
            const int grp = item / WC, k = item % WC;
            const int cls = k / (WC / 2), kk = k % (WC / 2);
            const int zl = kk / (P / 2), idx = kk % (P / 2);
            const int z = z0 + zl;
            const int typar = (cls ^ (z >> t_log2)) & 1;
            const int iw = ((2 * (idx >> w_log2) + typar) << w_log2) + (idx & wmask);
            const int wl = zl * P + iw;
            const int64_t wq = (int64_t)z * P + iw;
            // blocks in tiles of the visited coarse colour: tile x parity = coarse xor class
            const uint32_t amask = ((coarse ^ cls) & 1) ? mh.odd_tx : (~mh.odd_tx & 0xFFu);
            float4 hh4[8] = {};
            if (!BIM) {
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if ((amask >> j) & 1u) hh4[j] = __ldg(field4 + field4_index(c, wq, j, WPAD));
            }
            const uint32_t p0 = parity0_mask<L>(c, z, iw);
            uint32_t c0[GT], c1[GT], c2w[GT], sf[GT], flip[GT];
#pragma unroll
            for (int gg = 0; gg < GT; ++gg) {
              const int g = min(grp * GT + gg, gact - 1);
              uint32_t nb[6];
              neighbour_words<L, S>(sp + ((size_t)g * 2 + (c ^ 1)) * WC, zl, iw, p0, up_rank, dn_rank, nb);
              count6(nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], c0[gg], c1[gg], c2w[gg]);
              sf[gg] = sp[((size_t)g * 2 + c) * WC + wl];
              flip[gg] = 0u;
            }
            const uint32_t fb = BIM ? v.hbits[(int64_t)c * W + wq] : 0u;
            PairSlices ps[GT];
#pragma unroll
            for (int gg = 0; gg < GT; ++gg) ps[gg] = make_pairs(c0[gg], c1[gg], c2w[gg], sf[gg], fb);
            uint32_t fk[GT][4];
#pragma unroll
            for (int gg = 0; gg < GT; ++gg)
#pragma unroll
              for (int q = 0; q < 4; ++q) fk[gg][q] = 0u;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              const int j = 7 - jj;
              if ((amask >> j) & 1u) {
#pragma unroll
                for (int gg = 0; gg < GT; ++gg) {
                  const int g = min(grp * GT + gg, gact - 1);
                  const Words4 w = philox10(v.seed, v.realization, (uint32_t)(8 * wq + j), (uint32_t)(r0 + g), c2, tag);
                  decide_block<BIM>(w, ps[gg], j, slot0 + (uint32_t)g * kTabSlot, hh4[j], flip[gg], fk[gg]);
                }
              } else if (!BIM) {
                // keep block j's sign bits at bit j of fk: a skipped block shifts in zeros
#pragma unroll
                for (int gg = 0; gg < GT; ++gg)
#pragma unroll
                  for (int q = 0; q < 4; ++q) fk[gg][q] <<= 1;
              }
            }
            if (!BIM) {
#pragma unroll
              for (int gg = 0; gg < GT; ++gg)
                flip[gg] = fk[gg][0] | (fk[gg][1] << 8) | (fk[gg][2] << 16) | (fk[gg][3] << 24);
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
    }
  }

  for (int t = tid; t < gact * 2 * WC; t += nt) {
    const int g = t / (2 * WC), rem = t % (2 * WC), c = rem / WC, wl = rem % WC;
    v.bits[((int64_t)(r0 + g) * 2 + c) * W + (int64_t)z0 * P + wl] = sp[t];
  }
  if (xa.enabled) interval_tail<L, S, BIM>(v, G, r0, gact, rank, nsw, field4, xa);
}

template <int L, int S, int GT, bool BIM, int NT>
__global__ void __launch_bounds__(NT) k_sweeps_bits_mh(RealView v, int32_t G, uint32_t sweep0, int32_t nsw,
                                                        const float4 *__restrict__ field4, ExchArgs xa, MultiHit mh) {
  const int rank = S > 1 ? (int)cluster_rank() : 0;
  const int r0 = (int)(blockIdx.x / S) * G;
  const int gact = min(G, v.R - r0);
  xa.expected = gridDim.x;
  bits_interval_mh<L, S, GT, BIM>(v, G, r0, gact, rank, sweep0, nsw, field4, xa, mh);
}

}  // namespace rfim
