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
// to threads grouped by the parity of (y/T + z/T), so the 32 words of a warp update the same
// blocks; the tile edge is a template parameter, so which blocks is known at compile time.
#pragma once
#include <cstdint>

#include "kernels_bits.cuh"
#include "sweep_bits.h"

namespace rfim {

// Blocks j of a word (x in [8 j mod L, 8 j mod L + 8)) that lie in tiles of odd x index.
__host__ __device__ constexpr uint32_t odd_tile_blocks(int L, int T) {
  uint32_t m = 0u;
  for (int j = 0; j < 8; ++j)
    if ((((8 * j) % L) / T) & 1) m |= 1u << j;
  return m;
}

template <int L, int S, int GT, bool BIM, int T>
__device__ __forceinline__ void bits_interval_mh(const RealView &v, int G, int r0, int gact, int rank, uint32_t sweep0,
                                                 int nsw, const float4 *__restrict__ field4, const ExchArgs &xa,
                                                 const MultiHit &mh) {
  using Gm = BitsGeom<L>;
  constexpr int P = Gm::P, PZ = L / S, WC = PZ * P;
  constexpr int RW = 64 / L;  // rows of one colour held by a word
  static_assert(L >= 16 && WC % 64 == 0, "a warp's words must share one parity class");
  extern __shared__ __align__(16) uint32_t sm[];
  const int up_rank = (rank + 1) % S, dn_rank = (rank + S - 1) % S;
  const int z0 = rank * PZ;
  __syncthreads();
  uint32_t *sp = sm;
  uint32_t *tab = sm + (size_t)G * 2 * WC;
  const uint32_t slot0 = tab_slot0(tab);
  const int nt = blockDim.x, tid = threadIdx.x;

  copy_slab<L, S, true>(v, sp, r0, gact, z0);
  tab_fill<BIM>(v, tab, slot0, gact, [&](int g) { return r0 + g; });
  sync_slabs<S>();

  const int ngroups = (gact + GT - 1) / GT;
  const int items = WC * ngroups;
  // words of one tile band (T rows) in a plane; blocks in tiles of odd / even x index
  constexpr int WPT = T / RW;
  constexpr uint32_t ODD = odd_tile_blocks(L, T), EVEN = ~ODD & 0xFFu;
  static_assert(T % 8 == 0 && L % (2 * T) == 0 && WPT >= 1, "tiles of edge 8, 16 or 32 dividing L / 2");
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
            const int typar = (cls ^ (z / T)) & 1;
            const int iw = (2 * (idx / WPT) + typar) * WPT + idx % WPT;
            // blocks in tiles of the visited coarse colour: tile x parity = coarse xor class
            // (uniform over the warp, whose 32 words share the class)
            if ((coarse ^ cls) & 1)
              update_word<L, S, GT, BIM, ODD>(v, sp, c, zl, iw, z0, grp, gact, r0, c2, tag, slot0, field4, up_rank,
                                              dn_rank);
            else
              update_word<L, S, GT, BIM, EVEN>(v, sp, c, zl, iw, z0, grp, gact, r0, c2, tag, slot0, field4, up_rank,
                                               dn_rank);
          }
          sync_slabs<S>();
        }
      }
    }
  }

  copy_slab<L, S, false>(v, sp, r0, gact, z0);
  if (xa.enabled) interval_tail<L, S, BIM>(v, G, r0, gact, rank, nsw, field4, xa);
}

template <int L, int S, int GT, bool BIM, int NT, int T>
__global__ void __launch_bounds__(NT) k_sweeps_bits_mh(RealView v, int32_t G, uint32_t sweep0, int32_t nsw,
                                                        const float4 *__restrict__ field4, ExchArgs xa, MultiHit mh) {
  const int rank = S > 1 ? (int)cluster_rank() : 0;
  const int r0 = (int)(blockIdx.x / S) * G;
  const int gact = min(G, v.R - r0);
  xa.expected = gridDim.x;
  bits_interval_mh<L, S, GT, BIM, T>(v, G, r0, gact, rank, sweep0, nsw, field4, xa, mh);
}

}  // namespace rfim
