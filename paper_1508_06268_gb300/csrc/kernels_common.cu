// Set-up, energy, exchange and conversion kernels shared by both spin layouts.
#include <cmath>
#include <algorithm>
#include <cstdint>

#include "exchange.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "philox.cuh"

namespace rfim {

namespace {

constexpr int kThreads = 256;

__host__ __device__ inline int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 65535LL * 8) b = 65535LL * 8;
  return (int)b;
}

__device__ __forceinline__ int get_spin(const RealView &v, bool bitpack, int32_t r, int32_t c, int64_t q) {
  const int64_t half = (int64_t)v.N / 2;
  if (bitpack) {
    const uint32_t w = v.bits[((int64_t)r * 2 + c) * (half / 32) + (q >> 5)];
    return (int)((w >> bit_of(q)) & 1u);
  }
  return v.spins8[((int64_t)r * 2 + c) * half + q];
}

// Field realization (Sec. 3.1 step 2): unscaled h_i in natural order plus the scaled,
// colour-compacted copies the sweep kernels read.
__global__ void k_field(RealView v, int32_t kind, uint32_t field_seed, float h, float *hraw, float *hh_c,
                        uint8_t *hbit_c, uint32_t *hbits) {
  const int64_t N = v.N, half = N / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    float hv;
    if (kind == kBimodal) {
      const Words4 w = philox10(field_seed, v.realization, (uint32_t)(i >> 2), 0u, 0u, tag_word(kTagField, 0, 0));
      hv = (w.w[i & 3] >> 31) ? -1.0f : 1.0f;
      hraw[i] = hv;
    } else if (kind == kGaussian) {
      const Words4 w = philox10(field_seed, v.realization, (uint32_t)(i >> 1), 1u, 0u, tag_word(kTagField, 0, 0));
      const double u1 = ((double)w.w[2 * (i & 1)] + 0.5) * 0x1p-32;
      const double u2 = ((double)w.w[2 * (i & 1) + 1] + 0.5) * 0x1p-32;
      const double z = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
      hv = (float)z;
      hraw[i] = hv;
    } else {
      hv = hraw[i];  // explicit: uploaded by the host
    }
    const int32_t L = v.L;
    const int32_t x = (int32_t)(i % L), y = (int32_t)((i / L) % L), z = (int32_t)(i / ((int64_t)L * L));
    const int32_t c = (x + y + z) & 1;
    const int64_t q = q_of(L, v.Lh, x, y, z);
    hh_c[c * half + q] = __fmul_rn(h, hv);
    hbit_c[c * half + q] = hv > 0.0f ? 1 : 0;
  }
}

// Bit-layout copy of the field sign bits: one thread per word.
__global__ void k_field_bits(RealView v, const uint8_t *hbit_c, uint32_t *hbits) {
  const int64_t half = (int64_t)v.N / 2, words = half / 32;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * words; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / words, wd = t % words;
    uint32_t out = 0;
    for (int p = 0; p < 32; ++p) {
      const int64_t q = wd * 32 + p;
      out |= (uint32_t)hbit_c[c * half + q] << bit_of(q);
    }
    hbits[t] = out;
  }
}

// Random start (Sec. 3.1 step 3).
__global__ void k_init_int8(RealView v, int32_t R, uint32_t stage) {
  const int64_t N = v.N, half = N / 2, total = N * R;
  const int32_t L = v.L;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(t / N);
    const int64_t i = t % N;
    const Words4 w = philox10(v.seed, v.realization, (uint32_t)(i >> 2), (uint32_t)r, 0u, tag_word(kTagInit, stage, 0));
    const int32_t x = (int32_t)(i % L), y = (int32_t)((i / L) % L), z = (int32_t)(i / ((int64_t)L * L));
    const int32_t c = (x + y + z) & 1;
    v.spins8[((int64_t)r * 2 + c) * half + q_of(L, v.Lh, x, y, z)] = (w.w[i & 3] >> 31) ? 0 : 1;
  }
}

// Random start in the bit layout: one thread per destination word (all 32 sites of one colour).
__global__ void k_init_bits(RealView v, int32_t R, uint32_t stage) {
  const int64_t half = (int64_t)v.N / 2, words = half / 32, total = (int64_t)R * 2 * words;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(t / (2 * words));
    const int32_t c = (int32_t)((t / words) & 1);
    const int64_t wd = t % words;
    uint32_t out = 0;
    for (int p = 0; p < 32; ++p) {
      const int64_t q = wd * 32 + p;
      const Site s = site_of_q(v.L, v.Lh, c, q);
      const int64_t i = (int64_t)s.x + (int64_t)v.L * ((int64_t)s.y + (int64_t)v.L * s.z);
      const Words4 w = philox10(v.seed, v.realization, (uint32_t)(i >> 2), (uint32_t)r, 0u, tag_word(kTagInit, stage, 0));
      out |= (uint32_t)((w.w[i & 3] >> 31) ? 0u : 1u) << bit_of(q);
    }
    v.bits[t] = out;
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Energy (Eq. 1) of every replica: B over the 3N forward bonds equals the sum over colour-0
// sites of s_i times its six neighbours (every bond joins the two colours once; for L = 2 the
// doubled x-pairs appear twice in both forms).  One CTA per replica.
//   bimodal: F = h * (exact integer sum of h_i s_i), E exact in double
//   float field: sum of hh_i s_i accumulated error-free per thread (Ogita-Rump-Oishi Sum2 in
//   float: running sum plus the running sum of the exact TwoSum rounding errors), then in double.
__global__ void k_energy(RealView v, double J, double h, bool bitpack) {
  const int32_t r = blockIdx.x;
  const int32_t L = v.L, Lh = v.Lh;
  const int64_t half = (int64_t)v.N / 2;
  long long B = 0, M = 0, Fi = 0;
  float fs = 0.0f, fe = 0.0f;
  for (int32_t c = 0; c < 2; ++c) {
    for (int64_t q = threadIdx.x; q < half; q += blockDim.x) {
      const int si = 2 * get_spin(v, bitpack, r, c, q) - 1;
      M += si;
      if (c == 0) {
        const Site s = site_of_q(L, Lh, 0, q);
        int64_t nq[6];
        neighbour_qs(L, Lh, s, nq);
        int up = 0;
#pragma unroll
        for (int d = 0; d < 6; ++d) up += get_spin(v, bitpack, r, 1, nq[d]);
        B += si * (2 * up - 6);
      }
      if (v.kind == kBimodal) {
        Fi += si * (v.hbit_c[c * half + q] ? 1 : -1);
      } else {
        const float term = si > 0 ? v.hh_c[c * half + q] : -v.hh_c[c * half + q];
        const float t = __fadd_rn(fs, term);
        const float bp = __fsub_rn(t, fs);
        const float err = __fadd_rn(__fsub_rn(fs, __fsub_rn(t, bp)), __fsub_rn(term, bp));
        fs = t;
        fe = __fadd_rn(fe, err);
      }
    }
  }
  double F = (double)fs + (double)fe;
  __shared__ long long sB[32], sM[32], sF[32];
  __shared__ double sD[32];
  B = warp_sum(B);
  M = warp_sum(M);
  Fi = warp_sum(Fi);
  F = warp_sum(F);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
    sB[wid] = B;
    sM[wid] = M;
    sF[wid] = Fi;
    sD[wid] = F;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tb = 0, tm = 0, tf = 0;
    double td = 0.0;
    for (int w = 0; w < nw; ++w) {
      tb += sB[w];
      tm += sM[w];
      tf += sF[w];
      td += sD[w];
    }
    const double Fv = v.kind == kBimodal ? h * (double)tf : td;
    v.E[r] = -J * (double)tb - Fv;
    v.M[r] = tm;
  }
}

// The same energies for the int8 layout when L % 8 == 0, four sites per step: each neighbour
// direction of a group of four same-colour sites is one 32-bit word of 0/1 bytes (see the int8
// sweep), so s_i s_j summed over the group is 4 - 2 popc(self ^ neighbour word).  LC: the edge
// length when fixed at compile time, else 0.
template <int LC>
__global__ void k_energy_int8_rows(RealView v, double J, double h) {
  const int32_t r = blockIdx.x;
  const int32_t L = LC ? LC : v.L, Lh = L / 2;
  const int32_t half = L * L * Lh, plane = L * Lh, groups = half / 4;
  const uint8_t *S0 = v.spins8 + (int64_t)r * 2 * half, *S1 = S0 + half;
  auto ld = [](const uint8_t *p) { return *reinterpret_cast<const uint32_t *>(p); };
  long long B = 0, M = 0, Fi = 0;
  float fs = 0.0f, fe = 0.0f;
  for (int32_t c = 0; c < 2; ++c) {
    const uint8_t *S = c ? S1 : S0;
    for (int32_t g = threadIdx.x; g < groups; g += blockDim.x) {
      const int32_t q0 = 4 * g;
      const uint32_t self = ld(S + q0);
      M += 2 * __popc(self) - 4;
      if (c == 0) {
        const int32_t xh0 = q0 % Lh;
        const int32_t row = q0 / Lh;
        const int32_t y = row % L, z = row / L;
        const uint32_t par = (uint32_t)((y + z) & 1);
        const uint32_t w0 = ld(S1 + q0);
        const int32_t xa = par ? (xh0 + 4 == Lh ? 0 : xh0 + 4) : (xh0 == 0 ? Lh - 4 : xh0 - 4);
        const uint32_t wa = ld(S1 + (q0 - xh0) + xa);
        const uint32_t wx = par ? __byte_perm(w0, wa, 0x4321u) : __byte_perm(wa, w0, 0x6543u);
        const uint32_t wyp = ld(S1 + (y == L - 1 ? q0 + Lh - plane : q0 + Lh));
        const uint32_t wym = ld(S1 + (y == 0 ? q0 - Lh + plane : q0 - Lh));
        const uint32_t wzp = ld(S1 + (z == L - 1 ? q0 + plane - half : q0 + plane));
        const uint32_t wzm = ld(S1 + (z == 0 ? q0 - plane + half : q0 - plane));
        B += 24 - 2 * (__popc(self ^ w0) + __popc(self ^ wx) + __popc(self ^ wyp) + __popc(self ^ wym) +
                       __popc(self ^ wzp) + __popc(self ^ wzm));
      }
      if (v.kind == kBimodal) {
        Fi += 4 - 2 * __popc(self ^ ld(v.hbit_c + c * half + q0));
      } else {
        const float4 h4 = *reinterpret_cast<const float4 *>(v.hh_c + c * half + q0);
        const float hk[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float term = ((self >> (8 * j)) & 1u) ? hk[j] : -hk[j];
          const float t = __fadd_rn(fs, term);
          const float bp = __fsub_rn(t, fs);
          const float err = __fadd_rn(__fsub_rn(fs, __fsub_rn(t, bp)), __fsub_rn(term, bp));
          fs = t;
          fe = __fadd_rn(fe, err);
        }
      }
    }
  }
  double F = (double)fs + (double)fe;
  __shared__ long long sB[32], sM[32], sF[32];
  __shared__ double sD[32];
  B = warp_sum(B);
  M = warp_sum(M);
  Fi = warp_sum(Fi);
  F = warp_sum(F);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
    sB[wid] = B;
    sM[wid] = M;
    sF[wid] = Fi;
    sD[wid] = F;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tb = 0, tm = 0, tf = 0;
    double td = 0.0;
    for (int w = 0; w < nw; ++w) {
      tb += sB[w];
      tm += sM[w];
      tf += sF[w];
      td += sD[w];
    }
    const double Fv = v.kind == kBimodal ? h * (double)tf : td;
    v.E[r] = -J * (double)tb - Fv;
    v.M[r] = tm;
  }
}

// The same energies with eight sites per thread (64-bit words, L % 16 == 0) and each replica
// spread over gridDim.x CTAs of one grid row: partial sums per (replica, CTA), then the last CTA
// of the replica to arrive adds them in CTA order, so the result does not depend on which one
// that is.  B, M and the bimodal field count are exact integers; the float field term is an
// error-free running sum per thread (as above), added in double in a fixed order.
template <int LC>
__global__ void __launch_bounds__(256) k_energy_int8_rows8(RealView v, double J, double h, EnergyParts ep) {
  const int32_t r = blockIdx.y, part = blockIdx.x, nparts = gridDim.x;
  const int32_t L = LC ? LC : v.L, Lh = L / 2;
  const int32_t half = L * L * Lh, plane = L * Lh, groups = half / 8;
  const uint8_t *S0 = v.spins8 + (int64_t)r * 2 * half, *S1 = S0 + half;
  auto ld = [](const uint8_t *p) { return *reinterpret_cast<const uint64_t *>(p); };
  long long B = 0, M = 0, Fi = 0;
  float fs = 0.0f, fe = 0.0f;
  for (int32_t c = 0; c < 2; ++c) {
    const uint8_t *S = c ? S1 : S0;
    for (int32_t g = part * blockDim.x + threadIdx.x; g < groups; g += nparts * blockDim.x) {
      const int32_t q0 = 8 * g;
      const uint64_t self = ld(S + q0);
      M += 2 * __popcll(self) - 8;
      if (c == 0) {
        // colour-0 sites with their six colour-1 neighbours: every bond once
        const int32_t xh0 = q0 % Lh;
        const int32_t row = q0 / Lh;
        const int32_t y = row % L, z = row / L;
        const bool par = ((y + z) & 1) != 0;
        const uint64_t w0 = ld(S1 + q0);
        const int32_t xa = par ? (xh0 + 8 == Lh ? 0 : xh0 + 8) : (xh0 == 0 ? Lh - 8 : xh0 - 8);
        const uint64_t wa = ld(S1 + (q0 - xh0) + xa);
        const uint64_t wx = par ? ((w0 >> 8) | (wa << 56)) : ((w0 << 8) | (wa >> 56));
        const uint64_t wyp = ld(S1 + (y == L - 1 ? q0 + Lh - plane : q0 + Lh));
        const uint64_t wym = ld(S1 + (y == 0 ? q0 - Lh + plane : q0 - Lh));
        const uint64_t wzp = ld(S1 + (z == L - 1 ? q0 + plane - half : q0 + plane));
        const uint64_t wzm = ld(S1 + (z == 0 ? q0 - plane + half : q0 - plane));
        B += 48 - 2 * (__popcll(self ^ w0) + __popcll(self ^ wx) + __popcll(self ^ wyp) + __popcll(self ^ wym) +
                       __popcll(self ^ wzp) + __popcll(self ^ wzm));
      }
      if (v.kind == kBimodal) {
        Fi += 8 - 2 * __popcll(self ^ ld(v.hbit_c + c * half + q0));
      } else {
        const float4 *hp = reinterpret_cast<const float4 *>(v.hh_c + c * half + q0);
        const float4 ha = hp[0], hb = hp[1];
        const float hk[8] = {ha.x, ha.y, ha.z, ha.w, hb.x, hb.y, hb.z, hb.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float term = ((self >> (8 * j)) & 1u) ? hk[j] : -hk[j];
          const float t = __fadd_rn(fs, term);
          const float bp = __fsub_rn(t, fs);
          const float err = __fadd_rn(__fsub_rn(fs, __fsub_rn(t, bp)), __fsub_rn(term, bp));
          fs = t;
          fe = __fadd_rn(fe, err);
        }
      }
    }
  }
  double F = (double)fs + (double)fe;
  __shared__ long long sB[8], sM[8], sF[8];
  __shared__ double sD[8];
  B = warp_sum(B);
  M = warp_sum(M);
  Fi = warp_sum(Fi);
  F = warp_sum(F);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
    sB[wid] = B;
    sM[wid] = M;
    sF[wid] = Fi;
    sD[wid] = F;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tb = 0, tm = 0, tf = 0;
    double td = 0.0;
    for (int w = 0; w < nw; ++w) {
      tb += sB[w];
      tm += sM[w];
      tf += sF[w];
      td += sD[w];
    }
    const int64_t slot = (int64_t)r * kEnergyMaxParts + part;
    ep.B[slot] = tb;
    ep.M[slot] = tm;
    ep.Fi[slot] = tf;
    ep.F[slot] = td;
    __threadfence();
    if (atomicAdd(ep.count + r, 1u) == (unsigned)(nparts - 1)) {
      __threadfence();
      tb = tm = tf = 0;
      td = 0.0;
      for (int q = 0; q < nparts; ++q) {
        const int64_t s2 = (int64_t)r * kEnergyMaxParts + q;
        tb += __ldcg(ep.B + s2);
        tm += __ldcg(ep.M + s2);
        tf += __ldcg(ep.Fi + s2);
        td += __ldcg(ep.F + s2);
      }
      const double Fv = v.kind == kBimodal ? h * (double)tf : td;
      v.E[r] = -J * (double)tb - Fv;
      v.M[r] = tm;
      ep.count[r] = 0u;
    }
  }
}

// Structure factor F of the correlation length (Sec. 7; the spins s_i read for the printed h_i)
// of every replica, added to the accumulator of the replica's temperature after an exchange step:
// F = (1 / 3N) sum over the axes d of |sum_i s_i e^{i K i_d}|^2, K = 2 pi / L.  One CTA per
// replica: exact integer marginals S_d[t] = sum of the spins with coordinate t along axis d
// (shared-memory atomics), then the Fourier sums in double in a fixed order from tables
// cos(K t), sin(K t) computed on the host.
__global__ void k_measure_xi(RealView v, const double *kcos, const double *ksin, double *sumF, bool bitpack) {
  extern __shared__ int marg[];  // [3][L]
  const int32_t r = blockIdx.x, L = v.L, Lh = v.Lh;
  const int64_t half = (int64_t)v.N / 2;
  for (int t = threadIdx.x; t < 3 * L; t += blockDim.x) marg[t] = 0;
  __syncthreads();
  for (int32_t c = 0; c < 2; ++c) {
    for (int64_t q = threadIdx.x; q < half; q += blockDim.x) {
      const int si = 2 * get_spin(v, bitpack, r, c, q) - 1;
      const Site s = site_of_q(L, Lh, c, q);
      atomicAdd(&marg[s.x], si);
      atomicAdd(&marg[L + s.y], si);
      atomicAdd(&marg[2 * L + s.z], si);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0.0;
    for (int d = 0; d < 3; ++d) {
      double cs = 0.0, sn = 0.0;
      for (int t = 0; t < L; ++t) {
        cs = __dadd_rn(cs, __dmul_rn(kcos[t], (double)marg[d * L + t]));
        sn = __dadd_rn(sn, __dmul_rn(ksin[t], (double)marg[d * L + t]));
      }
      F = __dadd_rn(F, __dadd_rn(__dmul_rn(cs, cs), __dmul_rn(sn, sn)));
    }
    const int k = v.r2t[r];
    sumF[k] = __dadd_rn(sumF[k], F / (3.0 * (double)v.N));
  }
}

// The same marginals at L = 64, where a row (y, z) of one colour holds 32 sites, in-word site i at
// x = 2 i + ((colour + y + z) & 1) (bit layout: bit 8 (i & 3) + (i >> 2) of the row's word): a warp
// takes 32 rows at a time; for each in-word site a ballot over the rows gives the up spins of
// the two columns x = 2i and 2i + 1, counted by lane i; row and plane sums come from popcounts.
// INT8: the int8 layout at L = 64 (a row of one colour is 32 bytes of 0/1, site i at byte i),
// turned into the same 32-bit row words with in-word site i at bit i.
template <bool INT8>
__global__ void k_measure_xi_rows64(RealView v, const double *kcos, const double *ksin, double *sumF) {
  constexpr int L = 64, W = L * L * L / 64;  // rows (words) per colour
  __shared__ int marg[3 * L];
  const int32_t r = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int t = threadIdx.x; t < 3 * L; t += blockDim.x) marg[t] = 0;
  __syncthreads();
  int ax0 = 0, ax1 = 0;  // column sums of x = 2 lane and 2 lane + 1
  for (int blk = warp; blk < 2 * W / 32; blk += nwarps) {
    const int c = blk / (W / 32), wq = (blk % (W / 32)) * 32 + lane;
    uint32_t w = 0u;
    if (INT8) {
      const uint4 *row = reinterpret_cast<const uint4 *>(v.spins8 + ((int64_t)r * 2 + c) * (W * 32) + (int64_t)wq * 32);
      const uint4 a = row[0], b = row[1];
      const uint32_t q[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int t = 0; t < 8; ++t)
        w |= ((q[t] & 1u) | ((q[t] >> 7) & 2u) | ((q[t] >> 14) & 4u) | ((q[t] >> 21) & 8u)) << (4 * t);
    } else {
      w = v.bits[((int64_t)r * 2 + c) * W + wq];
    }
    const int y = wq & (L - 1), z = wq / L;
    const int rs = 2 * __popc(w) - 32;
    atomicAdd(&marg[L + y], rs);
    int zs = rs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zs += __shfl_xor_sync(0xffffffffu, zs, o);
    if (lane == 0) atomicAdd(&marg[2 * L + z], zs);  // the 32 rows share z
    const uint32_t odd = __ballot_sync(0xffffffffu, ((c + y + z) & 1) != 0);
    const int n_odd = __popc(odd), n_even = 32 - n_odd;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const uint32_t m = __ballot_sync(0xffffffffu, (w >> (INT8 ? i : 8 * (i & 3) + (i >> 2))) & 1u);
      if (lane == i) {
        ax0 += 2 * __popc(m & ~odd) - n_even;
        ax1 += 2 * __popc(m & odd) - n_odd;
      }
    }
  }
  atomicAdd(&marg[2 * lane], ax0);
  atomicAdd(&marg[2 * lane + 1], ax1);
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0.0;
    for (int d = 0; d < 3; ++d) {
      double cs = 0.0, sn = 0.0;
      for (int t = 0; t < L; ++t) {
        cs = __dadd_rn(cs, __dmul_rn(kcos[t], (double)marg[d * L + t]));
        sn = __dadd_rn(sn, __dmul_rn(ksin[t], (double)marg[d * L + t]));
      }
      F = __dadd_rn(F, __dadd_rn(__dmul_rn(cs, cs), __dmul_rn(sn, sn)));
    }
    const int k = v.r2t[r];
    sumF[k] = __dadd_rn(sumF[k], F / (3.0 * (double)v.N));
  }
}

// One exchange step j plus measurement (exchange.cuh), one CTA.
__global__ void k_exchange(RealView v, uint32_t j, int64_t measure_from) { exchange_and_measure(v, j, measure_from); }

__global__ void k_to_natural(RealView v, int32_t R, bool bitpack, int8_t *out) {
  const int64_t N = v.N, total = N * R;
  const int32_t L = v.L;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(t / N);
    const int64_t i = t % N;
    const int32_t x = (int32_t)(i % L), y = (int32_t)((i / L) % L), z = (int32_t)(i / ((int64_t)L * L));
    out[t] = get_spin(v, bitpack, r, (x + y + z) & 1, q_of(L, v.Lh, x, y, z)) ? 1 : -1;
  }
}

__global__ void k_from_natural_int8(RealView v, int32_t R, const int8_t *in) {
  const int64_t N = v.N, half = N / 2, total = N * R;
  const int32_t L = v.L;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(t / N);
    const int64_t i = t % N;
    const int32_t x = (int32_t)(i % L), y = (int32_t)((i / L) % L), z = (int32_t)(i / ((int64_t)L * L));
    v.spins8[((int64_t)r * 2 + ((x + y + z) & 1)) * half + q_of(L, v.Lh, x, y, z)] = in[t] > 0 ? 1 : 0;
  }
}

__global__ void k_from_natural_bits(RealView v, int32_t R, const int8_t *in) {
  const int64_t half = (int64_t)v.N / 2, words = half / 32, total = (int64_t)R * 2 * words;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(t / (2 * words));
    const int32_t c = (int32_t)((t / words) & 1);
    const int64_t wd = t % words;
    uint32_t out = 0;
    for (int p = 0; p < 32; ++p) {
      const int64_t q = wd * 32 + p;
      const Site s = site_of_q(v.L, v.Lh, c, q);
      const int64_t i = (int64_t)s.x + (int64_t)v.L * ((int64_t)s.y + (int64_t)v.L * s.z);
      out |= (uint32_t)(in[(int64_t)r * v.N + i] > 0 ? 1u : 0u) << bit_of(q);
    }
    v.bits[t] = out;
  }
}

}  // namespace

cudaError_t launch_field(const RealView &v, int32_t kind, uint32_t field_seed, float h, float *hraw, float *hh_c,
                         uint8_t *hbit_c, uint32_t *hbits, cudaStream_t st) {
  k_field<<<grid_for(v.N, kThreads), kThreads, 0, st>>>(v, kind, field_seed, h, hraw, hh_c, hbit_c, hbits);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || hbits == nullptr) return e;
  k_field_bits<<<grid_for(v.N / 32, kThreads), kThreads, 0, st>>>(v, hbit_c, hbits);
  return cudaGetLastError();
}

cudaError_t launch_init_spins(const RealView &v, int32_t R, uint32_t stage, bool bitpack, cudaStream_t st) {
  if (bitpack)
    k_init_bits<<<grid_for((int64_t)R * v.N / 32, kThreads), kThreads, 0, st>>>(v, R, stage);
  else
    k_init_int8<<<grid_for((int64_t)R * v.N, kThreads), kThreads, 0, st>>>(v, R, stage);
  return cudaGetLastError();
}

cudaError_t launch_energy(const RealView &v, double J, double h, bool bitpack, cudaStream_t st,
                          const EnergyParts *ep) {
  if (!bitpack && ep && v.L % 16 == 0 && (int64_t)v.N / 2 < ((int64_t)1 << 31)) {
    // about 2048 threads' worth of eight-site groups per CTA, at most kEnergyMaxParts CTAs per replica
    const int64_t groups = (int64_t)v.N / 16;
    const int parts = (int)std::min<int64_t>(kEnergyMaxParts, std::max<int64_t>(1, groups / 2048));
    const dim3 grid((unsigned)parts, (unsigned)v.R);
    switch (v.L) {
      case 16: k_energy_int8_rows8<16><<<grid, 256, 0, st>>>(v, J, h, *ep); break;
      case 32: k_energy_int8_rows8<32><<<grid, 256, 0, st>>>(v, J, h, *ep); break;
      case 64: k_energy_int8_rows8<64><<<grid, 256, 0, st>>>(v, J, h, *ep); break;
      default: k_energy_int8_rows8<0><<<grid, 256, 0, st>>>(v, J, h, *ep); break;
    }
    return cudaGetLastError();
  }
  if (!bitpack && v.L % 8 == 0 && (int64_t)v.N / 2 < ((int64_t)1 << 31)) {
    switch (v.L) {
      case 16: k_energy_int8_rows<16><<<v.R, 1024, 0, st>>>(v, J, h); break;
      case 32: k_energy_int8_rows<32><<<v.R, 1024, 0, st>>>(v, J, h); break;
      case 64: k_energy_int8_rows<64><<<v.R, 1024, 0, st>>>(v, J, h); break;
      default: k_energy_int8_rows<0><<<v.R, 1024, 0, st>>>(v, J, h); break;
    }
  } else
    k_energy<<<v.R, 512, 0, st>>>(v, J, h, bitpack);
  return cudaGetLastError();
}

cudaError_t launch_measure_xi(const RealView &v, const double *kcos, const double *ksin, double *sumF, bool bitpack,
                              cudaStream_t st) {
  if (v.L == 64 && bitpack)
    k_measure_xi_rows64<false><<<v.R, 512, 0, st>>>(v, kcos, ksin, sumF);
  else if (v.L == 64)
    k_measure_xi_rows64<true><<<v.R, 512, 0, st>>>(v, kcos, ksin, sumF);
  else
    k_measure_xi<<<v.R, 512, (size_t)3 * v.L * sizeof(int), st>>>(v, kcos, ksin, sumF, bitpack);
  return cudaGetLastError();
}

cudaError_t launch_exchange(const RealView &v, uint32_t j, int64_t measure_from, cudaStream_t st) {
  k_exchange<<<1, 256, 0, st>>>(v, j, measure_from);
  return cudaGetLastError();
}

cudaError_t launch_to_natural(const RealView &v, int32_t R, bool bitpack, int8_t *out, cudaStream_t st) {
  k_to_natural<<<grid_for((int64_t)R * v.N, kThreads), kThreads, 0, st>>>(v, R, bitpack, out);
  return cudaGetLastError();
}

cudaError_t launch_from_natural(const RealView &v, int32_t R, bool bitpack, const int8_t *in, cudaStream_t st) {
  if (bitpack)
    k_from_natural_bits<<<grid_for((int64_t)R * v.N / 32, kThreads), kThreads, 0, st>>>(v, R, in);
  else
    k_from_natural_int8<<<grid_for((int64_t)R * v.N, kThreads), kThreads, 0, st>>>(v, R, in);
  return cudaGetLastError();
}

}  // namespace rfim
