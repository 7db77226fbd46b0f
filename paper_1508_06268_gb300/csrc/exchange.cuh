// Exchange step and measurement, shared by the stand-alone exchange kernel and the fused tail of
// the bit-layout sweep kernel.  Runs inside one CTA; all its threads must call it.
#pragma once
#include <cstdint>

#include "internal.h"
#include "philox.cuh"

namespace rfim {

// Exchange step j (Eq. 2 read as W = min(1, e^Delta), Delta = (beta_k - beta_k+1)(E_a - E_b))
// over the disjoint pairs k = j mod 2, j mod 2 + 2, ... (odd xor even, Sec. 3.1 step 4),
// swapping temperature indices through t2r / r2t (Sec. 3.3), then, if j >= measure_from, one
// measurement per temperature of e = E/N, e^2, |m|, m^2, m^4 with m = M/N (Sec. 7).  With
// sumF set, also adds the structure factor Fr[r] of the replica now at each temperature to sumF
// (Fr written by other CTAs of this launch before their arrival, hence read through L2).  CG: the
// state was last written by another CTA of the same launch (several exchange steps per launch), so
// every load of it goes through L2, past this SM's L1.
template <bool CG = false>
__device__ __forceinline__ void exchange_and_measure(const RealView &v, uint32_t j, int64_t measure_from,
                                                     const double *Fr = nullptr, double *sumF = nullptr) {
  auto ld = [](const auto *p) { return CG ? __ldcg(p) : *p; };
  const int32_t R = v.R;
  for (int32_t p = threadIdx.x;; p += blockDim.x) {
    const int32_t k = (int32_t)(j & 1u) + 2 * p;
    if (k + 1 >= R) break;
    const int32_t a = ld(v.t2r + k), b = ld(v.t2r + k + 1);
    const double delta = (v.beta_d[k] - v.beta_d[k + 1]) * (ld(v.E + a) - ld(v.E + b));
    const Words4 w = philox10(v.seed, v.realization, (uint32_t)k, 0u, j, tag_word(kTagExch, v.stage, 0));
    const double u = (double)w.w[0] * 0x1p-32;
    const bool accept = (delta >= 0.0) || (u < exp(delta));
    v.att[k] = ld(v.att + k) + 1;
    if (accept) {
      v.acc[k] = ld(v.acc + k) + 1;
      v.t2r[k] = b;
      v.t2r[k + 1] = a;
      v.r2t[b] = k;
      v.r2t[a] = k + 1;
    }
  }
  __syncthreads();
  if ((int64_t)j >= measure_from) {
    const double Nd = (double)v.N;
    for (int32_t k = threadIdx.x; k < R; k += blockDim.x) {
      const int32_t a = ld(v.t2r + k);
      const double e = ld(v.E + a) / Nd;
      const double m = (double)ld(v.M + a) / Nd;
      // each product and sum rounded on its own (no fused multiply-add), as in the oracle
      double *acc = v.obs + (int64_t)k * 5;
      const double m2 = __dmul_rn(m, m);
      acc[0] = __dadd_rn(ld(acc + 0), e);
      acc[1] = __dadd_rn(ld(acc + 1), __dmul_rn(e, e));
      acc[2] = __dadd_rn(ld(acc + 2), fabs(m));
      acc[3] = __dadd_rn(ld(acc + 3), m2);
      acc[4] = __dadd_rn(ld(acc + 4), __dmul_rn(__dmul_rn(m2, m), m));
      if (sumF) sumF[k] = __dadd_rn(ld(sumF + k), __ldcg(Fr + a));
    }
    if (threadIdx.x == 0) *v.n_meas = ld(v.n_meas) + 1;
  }
  __syncthreads();
}

}  // namespace rfim
