// Metropolis acceptance tests shared by every sweep kernel, so that all spin layouts take
// identical decisions (Sec. 3.1 step 4; the paper does not print the rule: the standard
// min(1, exp(-beta dE)) is used, dE <= 0 accepted without a random number).
#pragma once
#include <cstdint>

namespace rfim {

// Bimodal field: the host tabulates thr = floor(exp(-beta dE) 2^32) clamped to [1, 2^32 - 1]
// for dE > 0 and stores thr - 1 (0xFFFFFFFF for dE <= 0), so the test is one unsigned compare.
__device__ __forceinline__ bool accept_table(uint32_t word, uint32_t thr_minus_one) {
  return word <= thr_minus_one;
}

__device__ __forceinline__ float ex2_approx(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

// Continuous field (Gaussian or explicit).  f = J n + hh_i in float (J n tabulated exactly as
// the float product), x = beta dE = (s 2 beta) f, which equals fl(beta * fl(2 s f)) because the
// factors 2 and s are exact.  Accept iff x <= 0 or u < exp(-x) with u = (word >> 8) 2^-24; the
// comparison is done as (word >> 8) < exp(-x) 2^24 in float (the left side is exact).
__device__ __forceinline__ bool accept_float(uint32_t word, float jn, float hh, float b2s) {
  const float f = __fadd_rn(jn, hh);
  const float x = __fmul_rn(b2s, f);
  const float p24 = __fmul_rn(ex2_approx(__fmul_rn(x, -1.44269504088896340736f)), 16777216.0f);
  const float k = __uint2float_rn(word >> 8);
  return !(x > 0.0f) || (k < p24);
}

}  // namespace rfim
