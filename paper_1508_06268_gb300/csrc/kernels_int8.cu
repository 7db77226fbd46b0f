// Checkerboard half-sweep on the int8 layout (any even L >= 2): the reference-shaped kernel.
// One thread updates the four consecutive same-colour sites q = 4g .. 4g+3 of one replica that
// share a Philox block (Sec. 3.1 step 4 Metropolis; Eq. 3 colours).  Neighbours are of the other
// colour, so every site sees the values from the start of the half-sweep.  Spins, field and
// tables are read from global memory (L2-resident for the sizes of interest).
#include <cstdint>

#include "decide.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "philox.cuh"

namespace rfim {

namespace {

template <bool kBimodalField>
__global__ void __launch_bounds__(256) k_halfsweep_int8(RealView v, int colour, uint32_t sweep) {
  const int32_t L = v.L, Lh = v.Lh;
  const int64_t half = (int64_t)v.N / 2, groups = half / 4, total = groups * v.R;
  const uint32_t tag = tag_word(kTagMetro, v.stage, (uint32_t)colour);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(t / groups);
    const int64_t g = t % groups;
    const int32_t k = v.r2t[r];
    uint8_t *self = v.spins8 + ((int64_t)r * 2 + colour) * half;
    const uint8_t *other = v.spins8 + ((int64_t)r * 2 + (colour ^ 1)) * half;
    const Words4 w = philox10(v.seed, v.realization, (uint32_t)g, (uint32_t)r, sweep, tag);
    uint32_t cur = *reinterpret_cast<const uint32_t *>(self + 4 * g);
    uint32_t nxt = cur;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t q = 4 * g + j;
      const Site s = site_of_q(L, Lh, colour, q);
      int64_t nq[6];
      neighbour_qs(L, Lh, s, nq);
      uint32_t up = 0;
#pragma unroll
      for (int d = 0; d < 6; ++d) up += other[nq[d]];
      const uint32_t sbit = (cur >> (8 * j)) & 1u;
      bool acc;
      if (kBimodalField) {
        const uint32_t idx = up | (sbit << 3) | ((uint32_t)v.hbit_c[colour * half + q] << 4);
        acc = accept_table(w.w[j], v.thr[(int64_t)k * 32 + idx]);
      } else {
        const float b2s = sbit ? v.b2l[k] : -v.b2l[k];
        acc = accept_float_l2e(w.w[j], v.gjn[up], v.hh_c[colour * half + q], b2s);
      }
      if (acc) nxt ^= 1u << (8 * j);
    }
    *reinterpret_cast<uint32_t *>(self + 4 * g) = nxt;
  }
}

}  // namespace

cudaError_t launch_halfsweep_int8(const RealView &v, int colour, uint32_t sweep, cudaStream_t st) {
  const int64_t total = (int64_t)v.N / 8 * v.R;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (v.kind == kBimodal)
    k_halfsweep_int8<true><<<(int)blocks, 256, 0, st>>>(v, colour, sweep);
  else
    k_halfsweep_int8<false><<<(int)blocks, 256, 0, st>>>(v, colour, sweep);
  return cudaGetLastError();
}

}  // namespace rfim
