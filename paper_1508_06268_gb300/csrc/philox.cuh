// Philox4x32-10 counter-based generator on the device, written from its published definition
// (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds,
// each multiplying words 0 and 2 by two odd constants (32x32 -> 64 bits) and mixing the high
// halves with words 1 and 3 and the round key; the key advances by two Weyl constants per round.
#pragma once
#include <cstdint>

namespace rfim {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Stream tags of the counter's word 3 (the paper names no generator; this keying makes every
// flip and exchange decision reproducible): c3 = (tag << 28) | (stage << 1) | colour.
constexpr uint32_t kTagInit = 1u, kTagMetro = 2u, kTagExch = 3u, kTagField = 4u;

__host__ __device__ __forceinline__ uint32_t tag_word(uint32_t tag, uint32_t stage, uint32_t colour) {
  return (tag << 28) | (stage << 1) | colour;
}

struct Words4 {
  uint32_t w[4];
};

__device__ __forceinline__ Words4 philox10(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                                           uint32_t c3) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    // one 32x32->64 multiply per product: the high and low halves come from the same instruction
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
    const uint32_t y0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t y2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = y0;
    c2 = y2;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  Words4 r;
  r.w[0] = c0;
  r.w[1] = c1;
  r.w[2] = c2;
  r.w[3] = c3;
  return r;
}

}  // namespace rfim
