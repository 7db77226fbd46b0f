// Checkerboard half-sweep on the int8 layout (Sec. 3.1 step 4 Metropolis; Eq. 3 colours).
// One thread updates the four consecutive same-colour sites q = 4g .. 4g+3 of one replica that
// share a Philox block.  Neighbours are of the other colour, so every site sees the values from
// the start of the half-sweep.  Spins and field are read from global memory (L2-resident for the
// sizes of interest).
//
// L % 8 == 0 (rows of L/2 sites hold whole groups of four): the four sites share y and z, so
// each neighbour direction is one 32-bit word of the other colour (x: the same word and a
// neighbouring word byte-shifted by one; y, z: the word L/2 or L^2/2 sites away, periodic).
// Spins are stored as 0/1 bytes, so the sum of the six words is the four up-counts, one per
// byte.  The decision table of the CTA's replica is in shared memory and addressed by one byte
// permute per site.  Other even L: one site at a time (k_halfsweep_int8).
#include <cstdint>

#include "decide.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "philox.cuh"

namespace rfim {

#ifndef RFIM_INT8_GT
#define RFIM_INT8_GT 8
#endif

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
        acc = accept_float_l2e(w.w[j], __fmul_rn(b2s, v.gjn[up]), v.hh_c[colour * half + q], b2s);
      }
      if (acc) nxt ^= 1u << (8 * j);
    }
    *reinterpret_cast<uint32_t *>(self + 4 * g) = nxt;
  }
}


__device__ __forceinline__ uint32_t ld_u32(const uint8_t *p) { return *reinterpret_cast<const uint32_t *>(p); }

// prmt.b32 in its default mode: a selector nibble with bit 3 set gives the sign of the selected
// byte replicated over the result byte.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

// Decisions of the four sites of one Philox block: 0/1 spin bytes `cur`, up-count bytes `up`,
// field bits `hb` (bimodal) or values `h4` (float), table slot `slot`.  Returns 0x01 in the byte
// of every accepted site.
template <bool kBimodalField>
__device__ __forceinline__ uint32_t decide4(const Words4 &w, uint32_t cur, uint32_t up, uint32_t hb, const float4 &h4,
                                            uint32_t slot) {
  if (kBimodalField) {
    const uint32_t offs = ((hb << 4) | (cur << 3) | up) << 2;  // per byte: table index x 4
    uint32_t flips = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t t;
      asm volatile("ld.shared.u32 %0, [%1];" : "=r"(t) : "r"(__byte_perm(offs, slot, 0x7650u | (uint32_t)j)));
      if (accept_table(w.w[j], t)) flips |= 1u << (8 * j);
    }
    return flips;
  }
  const float hk[4] = {h4.x, h4.y, h4.z, h4.w};
  const uint32_t offs = ((cur << 3) | up) << 3;  // per byte: table index x 8
  uint32_t sg[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 e;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(e.x), "=f"(e.y) : "r"(__byte_perm(offs, slot, 0x7650u | (uint32_t)j)));
    sg[j] = accept_float_sign(w.w[j], e.x, hk[j], e.y);
  }
  // byte j = 0xFF where site j is accepted (sign of the top byte of sg[j]), then one bit per byte
  const uint32_t m01 = prmt(sg[0], sg[1], 0x00FBu), m23 = prmt(sg[2], sg[3], 0xFB00u);
  return ((m01 & 0x0000FFFFu) | (m23 & 0xFFFF0000u)) & 0x01010101u;
}

// Per-replica decision tables of the CTA's GT replicas (64 words each: bimodal 32 x (thr - 1),
// float field 16 x (b J n, +-b)), filled by all threads.
template <bool kBimodalField, int GT>
__device__ __forceinline__ void int8_tables(const RealView &v, uint32_t *tab, int r0) {
  for (int t = threadIdx.x; t < GT * 32; t += blockDim.x) {
    const int gg = t >> 5, i = t & 31, r = min(r0 + gg, v.R - 1), k = v.r2t[r];
    if (kBimodalField) {
      tab[gg * 64 + i] = v.thr[(int64_t)k * 32 + i];
    } else if (i < 16) {
      const float b = (i >> 3) ? v.b2l[k] : -v.b2l[k];
      reinterpret_cast<float2 *>(tab + gg * 64)[i] = make_float2(__fmul_rn(b, v.gjn[i & 7]), b);
    }
  }
}

// grid: x over the groups of four sites, y over groups of GT replicas (GT temperature tables per
// CTA); a thread takes one group of four sites in GT replicas, which share the field load.
// LC: the edge length when fixed at compile time (index arithmetic by shifts, replica strides as
// address offsets), 0 for any L divisible by 8.
template <bool kBimodalField, int GT, int LC>
__global__ void __launch_bounds__(256) k_halfsweep_int8_rows(RealView v, int colour, uint32_t sweep) {
  __shared__ __align__(256) uint32_t tab[64 * GT];  // per replica a 256-byte slot
  const int32_t L = LC ? LC : v.L, Lh = L / 2;
  const int64_t half = (int64_t)L * L * Lh, plane = (int64_t)L * Lh;
  const int r0 = (int)blockIdx.y * GT;
  int8_tables<kBimodalField, GT>(v, tab, r0);
  __syncthreads();
  const int32_t g = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (g >= half / 4) return;
  const uint32_t slot0 = (uint32_t)__cvta_generic_to_shared(tab);
  const int32_t q0 = 4 * g;
  const int32_t xh0 = q0 % Lh;
  const int32_t row = q0 / Lh;
  const int32_t y = row % L, z = row / L;
  const bool odd = ((colour + y + z) & 1) != 0;
  // x neighbours: the same word, and the word before (even rows: site x - 1) or after (odd rows:
  // x + 1), periodic within the row, shifted by one byte; y, z: periodic rows and planes
  const int32_t qa = (q0 - xh0) + (odd ? (xh0 + 4 == Lh ? 0 : xh0 + 4) : (xh0 == 0 ? Lh - 4 : xh0 - 4));
  const int32_t yp = y == L - 1 ? q0 + Lh - (int32_t)plane : q0 + Lh;
  const int32_t ym = y == 0 ? q0 - Lh + (int32_t)plane : q0 - Lh;
  const int32_t zp = z == L - 1 ? q0 + (int32_t)plane - (int32_t)half : q0 + (int32_t)plane;
  const int32_t zm = z == 0 ? q0 - (int32_t)plane + (int32_t)half : q0 - (int32_t)plane;
  const uint32_t tag = tag_word(kTagMetro, v.stage, (uint32_t)colour);
  float4 h4 = make_float4(0.f, 0.f, 0.f, 0.f);
  uint32_t hb = 0u;
  if (kBimodalField)
    hb = ld_u32(v.hbit_c + colour * half + q0);
  else
    h4 = __ldg(reinterpret_cast<const float4 *>(v.hh_c + colour * half + q0));
  uint8_t *self0 = v.spins8 + ((int64_t)r0 * 2 + colour) * half;
  const uint8_t *O0 = v.spins8 + ((int64_t)r0 * 2 + (colour ^ 1)) * half;
#pragma unroll
  for (int gg = 0; gg < GT; ++gg) {
    const int r = r0 + gg;
    if (r >= v.R) break;
    uint8_t *self = self0 + 2 * half * gg;
    const uint8_t *O = O0 + 2 * half * gg;
    const uint32_t w0 = ld_u32(O + q0), wa = ld_u32(O + qa);
    const uint32_t wx = odd ? __byte_perm(w0, wa, 0x4321u) : __byte_perm(wa, w0, 0x6543u);
    const uint32_t up = w0 + wx + ld_u32(O + yp) + ld_u32(O + ym) + ld_u32(O + zp) + ld_u32(O + zm);
    const uint32_t cur = ld_u32(self + q0);
    const uint32_t slot = slot0 + 256u * gg;
    const Words4 w = philox10(v.seed, v.realization, (uint32_t)g, (uint32_t)r, sweep, tag);
    const uint32_t flips = decide4<kBimodalField>(w, cur, up, hb, h4, slot);
    *reinterpret_cast<uint32_t *>(self + q0) = cur ^ flips;
  }
}

__device__ __forceinline__ uint64_t ld_u64(const uint8_t *p) { return *reinterpret_cast<const uint64_t *>(p); }

// The same with eight consecutive same-colour sites (two Philox blocks) per thread and replica,
// for L % 16 == 0 (rows of L/2 sites hold whole groups of eight): each neighbour direction is one
// 64-bit load, so a site costs half the loads and index arithmetic of the four-site kernel.
template <bool kBimodalField, int GT, int LC>
__global__ void __launch_bounds__(256) k_halfsweep_int8_rows8(RealView v, int colour, uint32_t sweep) {
  __shared__ __align__(256) uint32_t tab[64 * GT];  // per replica a 256-byte slot
  const int32_t L = LC ? LC : v.L, Lh = L / 2;
  const int64_t half = (int64_t)L * L * Lh, plane = (int64_t)L * Lh;
  const int r0 = (int)blockIdx.y * GT;
  int8_tables<kBimodalField, GT>(v, tab, r0);
  __syncthreads();
  const int32_t g = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (g >= half / 8) return;
  const uint32_t slot0 = (uint32_t)__cvta_generic_to_shared(tab);
  const int32_t q0 = 8 * g;
  const int32_t xh0 = q0 % Lh;
  const int32_t row = q0 / Lh;
  const int32_t y = row % L, z = row / L;
  const bool odd = ((colour + y + z) & 1) != 0;
  // x neighbours: the same eight bytes and the group after (odd rows) or before (even rows),
  // periodic within the row, shifted by one byte; y, z: periodic rows and planes
  const int32_t qa = (q0 - xh0) + (odd ? (xh0 + 8 == Lh ? 0 : xh0 + 8) : (xh0 == 0 ? Lh - 8 : xh0 - 8));
  const int32_t yp = y == L - 1 ? q0 + Lh - (int32_t)plane : q0 + Lh;
  const int32_t ym = y == 0 ? q0 - Lh + (int32_t)plane : q0 - Lh;
  const int32_t zp = z == L - 1 ? q0 + (int32_t)plane - (int32_t)half : q0 + (int32_t)plane;
  const int32_t zm = z == 0 ? q0 - (int32_t)plane + (int32_t)half : q0 - (int32_t)plane;
  const uint32_t tag = tag_word(kTagMetro, v.stage, (uint32_t)colour);
  float4 h4a = make_float4(0.f, 0.f, 0.f, 0.f), h4b = h4a;
  uint64_t hb = 0u;
  if (kBimodalField) {
    hb = ld_u64(v.hbit_c + colour * half + q0);
  } else {
    const float4 *hp = reinterpret_cast<const float4 *>(v.hh_c + colour * half + q0);
    h4a = __ldg(hp);
    h4b = __ldg(hp + 1);
  }
  uint8_t *self0 = v.spins8 + ((int64_t)r0 * 2 + colour) * half;
  const uint8_t *O0 = v.spins8 + ((int64_t)r0 * 2 + (colour ^ 1)) * half;
#pragma unroll
  for (int gg = 0; gg < GT; ++gg) {
    const int r = r0 + gg;
    if (r >= v.R) break;
    uint8_t *self = self0 + 2 * half * gg;
    const uint8_t *O = O0 + 2 * half * gg;
    const uint64_t w0 = ld_u64(O + q0), wa = ld_u64(O + qa);
    const uint64_t wx = odd ? ((w0 >> 8) | (wa << 56)) : ((w0 << 8) | (wa >> 56));
    const uint64_t up = w0 + wx + ld_u64(O + yp) + ld_u64(O + ym) + ld_u64(O + zp) + ld_u64(O + zm);
    const uint64_t cur = ld_u64(self + q0);
    const uint32_t slot = slot0 + 256u * gg;
    const Words4 wl = philox10(v.seed, v.realization, (uint32_t)(2 * g), (uint32_t)r, sweep, tag);
    const Words4 wh = philox10(v.seed, v.realization, (uint32_t)(2 * g + 1), (uint32_t)r, sweep, tag);
    const uint32_t flo = decide4<kBimodalField>(wl, (uint32_t)cur, (uint32_t)up, (uint32_t)hb, h4a, slot);
    const uint32_t fhi = decide4<kBimodalField>(wh, (uint32_t)(cur >> 32), (uint32_t)(up >> 32),
                                                (uint32_t)(hb >> 32), h4b, slot);
    *reinterpret_cast<uint64_t *>(self + q0) = cur ^ ((uint64_t)fhi << 32 | flo);
  }
}

}  // namespace

cudaError_t launch_halfsweep_int8(const RealView &v, int colour, uint32_t sweep, cudaStream_t st) {
  if (v.L % 16 == 0 && (int64_t)v.N / 2 < ((int64_t)1 << 31)) {
    constexpr int GT = RFIM_INT8_GT;
    const int64_t groups = (int64_t)v.N / 16;
    const dim3 grid((unsigned)((groups + 255) / 256), (unsigned)((v.R + GT - 1) / GT));
    const bool bim = v.kind == kBimodal;
    auto go = [&](auto kb, auto kf) {
      (bim ? kb : kf)<<<grid, 256, 0, st>>>(v, colour, sweep);
    };
    switch (v.L) {
      case 16: go(k_halfsweep_int8_rows8<true, GT, 16>, k_halfsweep_int8_rows8<false, GT, 16>); break;
      case 32: go(k_halfsweep_int8_rows8<true, GT, 32>, k_halfsweep_int8_rows8<false, GT, 32>); break;
      case 64: go(k_halfsweep_int8_rows8<true, GT, 64>, k_halfsweep_int8_rows8<false, GT, 64>); break;
      default: go(k_halfsweep_int8_rows8<true, GT, 0>, k_halfsweep_int8_rows8<false, GT, 0>); break;
    }
    return cudaGetLastError();
  }
  if (v.L % 8 == 0 && (int64_t)v.N / 2 < ((int64_t)1 << 31)) {
    constexpr int GT = RFIM_INT8_GT;
    const int64_t groups = (int64_t)v.N / 8;
    const dim3 grid((unsigned)((groups + 255) / 256), (unsigned)((v.R + GT - 1) / GT));
    const bool bim = v.kind == kBimodal;
    auto go = [&](auto kb, auto kf) {
      (bim ? kb : kf)<<<grid, 256, 0, st>>>(v, colour, sweep);
    };
    switch (v.L) {
      case 16: go(k_halfsweep_int8_rows<true, GT, 16>, k_halfsweep_int8_rows<false, GT, 16>); break;
      case 32: go(k_halfsweep_int8_rows<true, GT, 32>, k_halfsweep_int8_rows<false, GT, 32>); break;
      case 64: go(k_halfsweep_int8_rows<true, GT, 64>, k_halfsweep_int8_rows<false, GT, 64>); break;
      default: go(k_halfsweep_int8_rows<true, GT, 0>, k_halfsweep_int8_rows<false, GT, 0>); break;
    }
    return cudaGetLastError();
  }
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
