// Instances of the bit-layout sweep kernel with split words (NS = 4): each 32-site word is updated
// by four warps, one pair of Philox blocks each (kernels_bits.cuh, split_unit).  For small
// lattices (L <= 32), whose half-sweeps hold too few words to keep the SMs issuing when one
// thread runs all eight blocks of a word.  One replica per unit (GT = 1).
#include "kernels_bits.cuh"
#include "sweep_bits.h"

namespace rfim {

namespace {
template <int L, int S, int NT>
void *pick_split(bool bim) {
  return bim ? (void *)k_sweeps_bits<L, S, 1, true, NT, false, 4> : (void *)k_sweeps_bits<L, S, 1, false, NT, false, 4>;
}
}  // namespace

void *kernel_for_split(int L, int S, int GT, int NT, bool bim) {
  if (GT != 1) return nullptr;
  if (L == 32 && S == 2 && NT == 1024) return pick_split<32, 2, 1024>(bim);
  if (L == 32 && S == 2 && NT == 512) return pick_split<32, 2, 512>(bim);
  if (L == 32 && S == 4 && NT == 512) return pick_split<32, 4, 512>(bim);
  if (L == 16 && S == 1 && NT == 1024) return pick_split<16, 1, 1024>(bim);
  if (L == 16 && S == 1 && NT == 512) return pick_split<16, 1, 512>(bim);
  if (L == 8 && S == 1 && NT == 512) return pick_split<8, 1, 512>(bim);
  if (L == 8 && S == 1 && NT == 256) return pick_split<8, 1, 256>(bim);
  return nullptr;
}

}  // namespace rfim
