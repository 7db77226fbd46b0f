// Internal declarations shared by the translation units of librfim (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

namespace rfim {

enum FieldKind : int32_t { kBimodal = 0, kGaussian = 1, kExplicit = 2 };

// Device-side view of one disorder realization.  All arrays are device pointers.
//   spins8  : int8 layout, uint8[Rcap][2][N/2], 1 = up, colour-compacted (q index within colour)
//   bits    : bit layout,  uint32[Rcap][2][N/64], colour-compacted, bit order within a word: the
//             site with in-word position p = 4j + k (j = 0..7, k = 0..3) sits at bit 8k + j
//   hh_c    : float[2][N/2] scaled field hh_i, colour-compacted
//   hbit_c  : uint8[2][N/2] 1 where h_i > 0 (bimodal tables)
//   hbits   : uint32[2][N/64] same as hbit_c in the bit layout
//   thr     : uint32[Rcap][32] bimodal acceptance thresholds minus one, per temperature index,
//             indexed by (#up neighbours | spin << 3 | field bit << 4); accept iff word <= thr
//   gjn     : float[8] J * (2u - 6) for u up neighbours (u = 7 unused)
//   b2      : float[Rcap] 2 * (float)beta_k
//   b2l     : float[Rcap] -2 * (float)beta_k * log2(e) rounded to float (bit-layout tables)
//   beta_d  : double[Rcap] beta_k = 1 / T_k
struct RealView {
  int32_t L, Lh, N, R;
  int32_t kind;
  uint32_t seed, realization, stage;
  uint8_t *spins8;
  uint32_t *bits;
  const float *hh_c;
  const uint8_t *hbit_c;
  const uint32_t *hbits;
  const uint32_t *thr;
  const float *gjn;
  const float *b2;
  const float *b2l;
  const double *beta_d;
  int32_t *t2r, *r2t;
  double *E;
  int64_t *M;
  uint64_t *att, *acc;
  double *obs;
  int64_t *n_meas;
};

// rfim_api.cu: records msg as the calling thread's last error (rfim_last_error(NULL)); returns code
int set_thread_error(int code, const std::string &msg);

// kernels_bits.cu: raises a kernel's dynamic shared-memory limit on the current device to at least
// `bytes`, never lowering it: contexts and servers with different shapes share the same kernels,
// and a smaller limit set by a later one would make the earlier one's launches fail.
cudaError_t raise_smem_limit(const void *fn, size_t bytes);

// host_tables.cu: bimodal thresholds (thr - 1, 32 entries per temperature), b2 = 2 beta,
// b2l = -2 beta log2 e, beta = 1/T, gjn[u] = J (2u - 6)
void bimodal_row(double beta, float J, float h, uint32_t out[32]);
void temperature_tables(const double *T, int32_t R, float J, float h, uint32_t *thr, float *b2, float *b2l,
                        double *beta, float gjn[8]);
// cos(K t), sin(K t) for t < L, K = 2 pi / L (the wave number of the Sec. 7 structure factor)
void wave_tables(int32_t L, double *kcos, double *ksin);

// kernels_common.cu
cudaError_t launch_field(const RealView &v, int32_t kind, uint32_t field_seed, float h, float *hraw,
                         float *hh_c, uint8_t *hbit_c, uint32_t *hbits, cudaStream_t st);
cudaError_t launch_init_spins(const RealView &v, int32_t R, uint32_t stage, bool bitpack, cudaStream_t st);
cudaError_t launch_exchange(const RealView &v, uint32_t j, int64_t measure_from, cudaStream_t st);
// Adds each replica's structure factor F (Sec. 7 correlation length) to sumF[r2t[r]].
cudaError_t launch_measure_xi(const RealView &v, const double *kcos, const double *ksin, double *sumF, bool bitpack,
                              cudaStream_t st);
cudaError_t launch_to_natural(const RealView &v, int32_t R, bool bitpack, int8_t *out, cudaStream_t st);
cudaError_t launch_from_natural(const RealView &v, int32_t R, bool bitpack, const int8_t *in, cudaStream_t st);
// Per-(replica, CTA) partial sums of the multi-CTA int8 energy reduction, owned by the caller:
// B, M, Fi, F [R][kEnergyMaxParts], arrival counters [R] (zero between launches).
constexpr int kEnergyMaxParts = 16;
struct EnergyParts {
  long long *B, *M, *Fi;
  double *F;
  unsigned int *count;
};
// E and M of every replica (Eq. 1) into v.E, v.M.  With ep (int8 layout, L % 16 == 0) the
// reduction spreads each replica over several CTAs; the last to arrive adds the partials in a
// fixed order.
cudaError_t launch_energy(const RealView &v, double J, double h, bool bitpack, cudaStream_t st,
                          const EnergyParts *ep = nullptr);

// kernels_int8.cu
cudaError_t launch_halfsweep_int8(const RealView &v, int colour, uint32_t sweep, cudaStream_t st);

}  // namespace rfim
