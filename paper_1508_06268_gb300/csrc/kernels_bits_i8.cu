// Instances of the bit-layout sweep kernel for realizations stored in the int8 layout: the slab
// of each CTA is packed from 0/1 bytes into bits in shared memory at the start of a launch and
// unpacked back at its end (kernels_bits.cuh, I8), so the int8 layout runs the same sweep,
// energy and exchange arithmetic as the bit layout.  Default cluster shapes of each L only (at L = 64 also one replica per thread, for R < 4).
#include "kernels_bits.cuh"
#include "sweep_bits.h"

namespace rfim {

namespace {
template <int L, int S, int GT, int NT>
void *pick_i8(bool bim) {
  return bim ? (void *)k_sweeps_bits<L, S, GT, true, NT, true> : (void *)k_sweeps_bits<L, S, GT, false, NT, true>;
}
}  // namespace

void *kernel_for_i8(int L, int S, int GT, int NT, bool bim) {
  if (L == 64 && S == 4 && GT == 4 && NT == 512) return pick_i8<64, 4, 4, 512>(bim);
  if (L == 64 && S == 4 && GT == 1 && NT == 512) return pick_i8<64, 4, 1, 512>(bim);  // R < 4
  if (L == 32 && S == 2 && GT == 1 && NT == 256) return pick_i8<32, 2, 1, 256>(bim);
  if (L == 16 && S == 1 && GT == 1 && NT == 512) return pick_i8<16, 1, 1, 512>(bim);
  if (L == 8 && S == 1 && GT == 1 && NT == 128) return pick_i8<8, 1, 1, 128>(bim);
  return nullptr;
}

}  // namespace rfim
