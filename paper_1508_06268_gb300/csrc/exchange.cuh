// Exchange step and measurement, shared by the stand-alone exchange kernel and the fused tail of
// the bit-layout sweep kernel.  Runs inside one CTA; all its threads must call it.
#pragma once
#include <cstdint>

#include "internal.h"
#include "philox.cuh"

namespace rfim {

// Swap decision of pair k at exchange step j (Eq. 2 read as W = min(1, e^Delta),
// Delta = (beta_k - beta_k+1)(E_a - E_b)), with Ea, Eb the energies of the replicas at
// temperatures k and k + 1.
__device__ __forceinline__ bool exchange_accept(const RealView &v, uint32_t j, int32_t k, double Ea, double Eb) {
  const double delta = (v.beta_d[k] - v.beta_d[k + 1]) * (Ea - Eb);
  const Words4 w = philox10(v.seed, v.realization, (uint32_t)k, 0u, j, tag_word(kTagExch, v.stage, 0));
  const double u = (double)w.w[0] * 0x1p-32;
  return (delta >= 0.0) || (u < exp(delta));
}

// One measurement (Sec. 7) of the replica at temperature k with energy E and magnetisation M:
// e = E/N, e^2, |m|, m^2, m^4 added to acc[0..4], each product and sum rounded on its own (no
// fused multiply-add), as in the oracle.
__device__ __forceinline__ void measure_add(double *acc, double E, int64_t M, double Nd) {
  const double e = E / Nd;
  const double m = (double)M / Nd;
  const double m2 = __dmul_rn(m, m);
  acc[0] = __dadd_rn(acc[0], e);
  acc[1] = __dadd_rn(acc[1], __dmul_rn(e, e));
  acc[2] = __dadd_rn(acc[2], fabs(m));
  acc[3] = __dadd_rn(acc[3], m2);
  acc[4] = __dadd_rn(acc[4], __dmul_rn(__dmul_rn(m2, m), m));
}

// Exchange step j over the disjoint pairs k = j mod 2, j mod 2 + 2, ... (odd xor even, Sec. 3.1
// step 4), swapping temperature indices through t2r / r2t (Sec. 3.3), then, if j >= measure_from,
// one measurement per temperature.  With sumF set, also adds the structure factor Fr[r] of the
// replica now at each temperature to sumF (Fr written by other CTAs of this launch before their
// arrival, hence read through L2).
__device__ __forceinline__ void exchange_and_measure(const RealView &v, uint32_t j, int64_t measure_from,
                                                     const double *Fr = nullptr, double *sumF = nullptr) {
  const int32_t R = v.R;
  for (int32_t p = threadIdx.x;; p += blockDim.x) {
    const int32_t k = (int32_t)(j & 1u) + 2 * p;
    if (k + 1 >= R) break;
    const int32_t a = v.t2r[k], b = v.t2r[k + 1];
    const bool accept = exchange_accept(v, j, k, v.E[a], v.E[b]);
    v.att[k] += 1;
    if (accept) {
      v.acc[k] += 1;
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
      const int32_t a = v.t2r[k];
      measure_add(v.obs + (int64_t)k * 5, v.E[a], v.M[a], Nd);
      if (sumF) sumF[k] = __dadd_rn(sumF[k], __ldcg(Fr + a));
    }
    if (threadIdx.x == 0) *v.n_meas += 1;
  }
  __syncthreads();
}

}  // namespace rfim
