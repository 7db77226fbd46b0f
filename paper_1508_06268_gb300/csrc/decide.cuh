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

// Continuous field (Gaussian or explicit).  The table carries b = fl(-2 beta log2 e) signed by the
// spin and bjn = fl(b J n); the exponent is t = fma(b, hh_i, bjn), one rounding of
// b (J n + hh_i) = -beta dE log2 e, so 2^t = exp(-beta dE) up to the roundings of b, bjn and t.
// The plain rule is: accept iff dE <= 0 or u < exp(-beta dE) with u = (word >> 8) 2^-24.  Here it
// is evaluated as rz(word) < 2^t 2^32, where rz(word) is the word rounded toward zero to a float
// (exactly 256 (word >> 8) for words >= 2^31, at most 128 above it otherwise).  t has the sign of
// -dE except where J n + hh_i cancels to within a rounding of bjn (|J n + hh_i| below about
// 2^-24 |J n|); for t >= 0, ex2.approx(t) >= 1 (checked over every float in [0, 1) on GB300), so
// the right side is >= 2^32 while rz(word) < 2^32: accepted, as the rule says.  For dE > 0 the
// threshold differs from the double-precision one by a few 2^-23 relative (ex2.approx and the
// float roundings), and a decision can differ only when u lands that close.
__device__ __forceinline__ float boltzmann_exponent(float bjn, float hh, float b) { return __fmaf_rn(b, hh, bjn); }

__device__ __forceinline__ bool accept_float_l2e(uint32_t word, float bjn, float hh, float b) {
  const float p32 = __fmul_rn(ex2_approx(boltzmann_exponent(bjn, hh, b)), 4294967296.0f);
  return __uint2float_rz(word) < p32;
}

// The same test as a sign bit: bit 31 of the result is 1 iff the move is accepted.  One FMA
// forms rz(word) - 2^t 2^32 with a single rounding; the product is exact (a power-of-two scaling)
// so the result is the correctly rounded difference, negative exactly when rz(word) < p32 and
// +0 when they are equal.
__device__ __forceinline__ uint32_t accept_float_sign(uint32_t word, float bjn, float hh, float b) {
  return __float_as_uint(__fmaf_rn(ex2_approx(boltzmann_exponent(bjn, hh, b)), -4294967296.0f, __uint2float_rz(word)));
}

}  // namespace rfim
