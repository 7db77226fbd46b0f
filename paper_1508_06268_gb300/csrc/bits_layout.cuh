// Word-level neighbour arithmetic of the bit layout (multi-spin coding), host and device.
//
// Layout: for colour c the N/2 sites are ordered by q = (x >> 1) + (L/2)(y + L z) and packed
// 32 per word; word wq = q >> 5 = z P + iw with P = L^2/64 words per plane.  Inside a word the
// site with position p = 4j + k (j = 0..7 "chunk", k = 0..3) is stored at bit 8k + j, so the four
// sites that share one Philox block are bit j of the four bytes: (word >> j) & 0x01010101.
// Rows have L/2 sites = g = L/8 chunks; for L < 64 a word holds 64/L whole rows, for L = 64 one.
//
// Every neighbour of a colour-c site is a colour-(1-c) site; for the 32 sites of a word the six
// neighbour bits form six words of the other colour:
//   A  same (y, z) row, same q                                   -> x+1 or x-1 depending on row parity
//   B  same row, q - 1 (row parity 0) or q + 1 (row parity 1)   -> the other x neighbour
//   C  y + 1 (q + L/2 within the plane, cyclic)
//   D  y - 1
//   E  z + 1 (same in-plane word)
//   F  z - 1
// with row parity (c + y + z) mod 2 (Eq. 3): for parity 0, x = 2 xh and the other colour holds
// x - 1 at xh - 1 and x + 1 at xh; for parity 1, x - 1 at xh and x + 1 at xh + 1.
#pragma once
#include <cstdint>

namespace rfim {

template <int L>
struct BitsGeom {
  static_assert(L == 8 || L == 16 || L == 32 || L == 64, "bit layout: L in {8,16,32,64}");
  static constexpr int Lh = L / 2;
  static constexpr int P = L * L / 64;          // words per plane per colour
  static constexpr int W = L * L * L / 64;      // words per colour
  static constexpr int G = L / 8;               // chunks per row (bits per row in each byte)
  // bits (of every byte) belonging to rows with the same parity as the word's first row
  static constexpr uint32_t kRowMask = L == 8 ? 0x55555555u : L == 16 ? 0x33333333u : L == 32 ? 0x0F0F0F0Fu : 0xFFFFFFFFu;
  // first and last bit of each row group inside a byte
  static constexpr uint32_t kGroupLo = L == 8 ? 0xFFu : L == 16 ? 0x55u : L == 32 ? 0x11u : 0x01u;
  static constexpr uint32_t kGroupHi = L == 8 ? 0xFFu : L == 16 ? 0xAAu : L == 32 ? 0x88u : 0x80u;
};

// Site at q - 1 within its row (cyclic) for every site of the word.
template <int L>
__host__ __device__ __forceinline__ uint32_t nb_minus1(uint32_t w) {
  using Gm = BitsGeom<L>;
  const uint32_t b3 = w >> 24;
  const uint32_t rot = ((b3 << 1) & ~Gm::kGroupLo & 0xFFu) | ((b3 >> (Gm::G - 1)) & Gm::kGroupLo);
  return (w << 8) | rot;
}

// Site at q + 1 within its row (cyclic) for every site of the word.
template <int L>
__host__ __device__ __forceinline__ uint32_t nb_plus1(uint32_t w) {
  using Gm = BitsGeom<L>;
  const uint32_t b0 = w & 0xFFu;
  const uint32_t rot = ((b0 >> 1) & ~Gm::kGroupHi & 0xFFu) | ((b0 << (Gm::G - 1)) & Gm::kGroupHi);
  return (w >> 8) | (rot << 24);
}

// Chunks [t, t + 8) of the 16-chunk concatenation (lo: chunks 0..7, hi: chunks 8..15), 0 < t < 8.
__host__ __device__ __forceinline__ uint32_t shift_chunks(uint32_t lo, uint32_t hi, int t) {
  const uint32_t keep = 0x01010101u * ((1u << (8 - t)) - 1u);
  return ((lo >> t) & keep) | ((hi << (8 - t)) & ~keep);
}

// Row-parity mask: bits of the word whose row has parity 0 (these take B = minus1(A)).
template <int L>
__host__ __device__ __forceinline__ uint32_t parity0_mask(int colour, int z, int iw) {
  const int y0 = L == 64 ? iw : iw * (64 / L);
  return ((colour + y0 + z) & 1) ? ~BitsGeom<L>::kRowMask : BitsGeom<L>::kRowMask;
}

// x and y neighbour words of in-plane word iw from the other colour's plane words.
//   same: word iw of the plane; next/prev: words (iw +- 1) mod P of the same plane
template <int L>
__host__ __device__ __forceinline__ void nb_xy(uint32_t same, uint32_t next, uint32_t prev, uint32_t p0mask,
                                               uint32_t &A, uint32_t &B, uint32_t &C, uint32_t &D) {
  A = same;
  B = (nb_minus1<L>(same) & p0mask) | (nb_plus1<L>(same) & ~p0mask);
  if (L == 64) {
    C = next;
    D = prev;
  } else {
    constexpr int t = BitsGeom<L>::G;  // one row = g chunks
    C = shift_chunks(same, next, t);
    D = shift_chunks(prev, same, 8 - t);
  }
}

// Bit-sliced count of up neighbours (0..6) for 32 sites: cnt = c0 + 2 c1 + 4 c2.
__host__ __device__ __forceinline__ void count6(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e, uint32_t f,
                                                uint32_t &c0, uint32_t &c1, uint32_t &c2) {
  const uint32_t s1 = a ^ b ^ c, k1 = (a & b) | (c & (a ^ b));
  const uint32_t s2 = d ^ e ^ f, k2 = (d & e) | (f & (d ^ e));
  c0 = s1 ^ s2;
  const uint32_t t = s1 & s2;
  c1 = k1 ^ k2 ^ t;
  c2 = (k1 & k2) | (t & (k1 ^ k2));
}

}  // namespace rfim
