// Lattice index helpers shared by the kernels.
//   natural site index   i = x + L (y + L z)
//   colour (Eq. 3)       c = (x + y + z) mod 2
//   index within colour  q = (x >> 1) + (L/2) (y + L z)   (unique: for fixed (y, z) the sites of
//                        colour c have x = 2 (x >> 1) + ((c + y + z) & 1))
//   bit layout           word q >> 5, bit 8 (q & 3) + ((q & 31) >> 2): the four sites drawn from
//                        one Philox block (q >> 2) sit at the same bit of the four bytes
#pragma once
#include <cstdint>

namespace rfim {

struct Site {
  int32_t x, y, z;
};

__host__ __device__ __forceinline__ Site site_of_q(int32_t L, int32_t Lh, int32_t colour, int64_t q) {
  const int32_t xh = (int32_t)(q % Lh);
  const int64_t t = q / Lh;
  const int32_t y = (int32_t)(t % L);
  const int32_t z = (int32_t)(t / L);
  Site s;
  s.x = 2 * xh + ((colour + y + z) & 1);
  s.y = y;
  s.z = z;
  return s;
}

__host__ __device__ __forceinline__ int64_t q_of(int32_t L, int32_t Lh, int32_t x, int32_t y, int32_t z) {
  return (int64_t)(x >> 1) + (int64_t)Lh * ((int64_t)y + (int64_t)L * z);
}

__host__ __device__ __forceinline__ int32_t bit_of(int64_t q) {
  return 8 * (int32_t)(q & 3) + (int32_t)((q & 31) >> 2);
}

// The six periodic neighbours of a site (all of the other colour), as q indices.
__host__ __device__ __forceinline__ void neighbour_qs(int32_t L, int32_t Lh, Site s, int64_t nq[6]) {
  const int32_t xp = s.x + 1 == L ? 0 : s.x + 1, xm = s.x == 0 ? L - 1 : s.x - 1;
  const int32_t yp = s.y + 1 == L ? 0 : s.y + 1, ym = s.y == 0 ? L - 1 : s.y - 1;
  const int32_t zp = s.z + 1 == L ? 0 : s.z + 1, zm = s.z == 0 ? L - 1 : s.z - 1;
  nq[0] = q_of(L, Lh, xp, s.y, s.z);
  nq[1] = q_of(L, Lh, xm, s.y, s.z);
  nq[2] = q_of(L, Lh, s.x, yp, s.z);
  nq[3] = q_of(L, Lh, s.x, ym, s.z);
  nq[4] = q_of(L, Lh, s.x, s.y, zp);
  nq[5] = q_of(L, Lh, s.x, s.y, zm);
}

}  // namespace rfim
