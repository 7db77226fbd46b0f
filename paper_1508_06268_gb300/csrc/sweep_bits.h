// Launch plan and launcher of the bit-layout sweep kernel.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"

namespace rfim {

struct FieldQuant;  // kernels_bits.cuh

// How one realization is mapped onto CTAs: a cluster of S CTAs (z slabs of L/S planes each)
// holds G replicas; every thread updates a word of the slab for GT of them at once (so one field
// load serves GT replicas).  Grid = ceil(R / G) clusters.  S == 0 selects the grid-wide
// cooperative kernel (kernels_grid.cuh): groups of 4 replicas, planes spread over one CTA per SM.
struct BitsPlan {
  int32_t L = 0, S = 1, G = 1, GT = 1, threads = 256;
  size_t smem = 0;
  int32_t Rcap = 0;
  float4 *field4 = nullptr;  // float path: hh as float4 per (colour, word, chunk), see kernels_bits.cu
  // float path: fixed-point field of the energy tail (flimb_index layout) and its exponent/sum
  uint4 *flimb = nullptr;
  FieldQuant *fquant = nullptr;
  // fused exchange tail: per-(replica, slab) partials and the arrival counter
  long long *partB = nullptr, *partM = nullptr, *partFi = nullptr;
  double *partF = nullptr;
  unsigned int *counter = nullptr;
  // grid-wide plan (S == 0): per-(replica, slab) partials, per-CTA progress words, SM count
  long long *gpartB = nullptr, *gpartM = nullptr, *gpartFi = nullptr;
  double *gpartF = nullptr;
  unsigned int *prog = nullptr;
  uint32_t *gbits = nullptr;  // int8 layout on the grid-wide plan: published end planes as bits
  // progress count the grid-wide kernel's words held when the next launch starts (each launch
  // adds its half-sweeps, so no launch has to zero them first)
  mutable uint32_t prog_base = 0;
  mutable uint32_t arrive_base = 0;  // the same for the arrival count of the exchange steps (counter[2])
  int32_t sms = 0;
  bool i8 = false;  // the realization is stored in the int8 layout and staged as bits (cluster shapes)
  int32_t NS = 1;   // 4: every word split over four warps, one block pair each (small lattices)
};

// Multi-hit double 3D checkerboard (Sec. 3.2, kernels_mh.cuh): mh local passes per tile visit
// (0: the plain checkerboard), tiles of edge `tile` (8, 16 or 32, dividing L / 2; the kernel is
// instantiated per tile edge).
struct MultiHit {
  int32_t mh = 0, tile = 0;
};
// Whether tiles of edge `tile` are supported at L; the setting for (L, mh, tile).
bool multihit_tile_ok(int32_t L, int32_t tile);
MultiHit make_multihit(int32_t L, int32_t mh, int32_t tile);
// Whether the plan's shape has a multi-hit instance; sets its launch attributes.
cudaError_t prepare_multihit(const BitsPlan &plan, bool bimodal);

bool bits_supported(int32_t L);
// Launch-shape tuner support: a thread-local candidate shape for the next make_bits_plan, the
// remembered best shape per (L, R, field kind), and the candidates instantiated for each L.
void set_plan_override(const char *plan);
void remember_tuned_plan(int32_t L, int32_t R, bool bimodal, const std::string &plan);
std::vector<std::string> plan_candidates(int32_t L);
int make_bits_plan(int32_t L, int32_t Rcap, bool bimodal, BitsPlan *plan, std::string *err, bool i8 = false);
// The int8-layout staging instance for a cluster shape (kernels_bits_i8.cu), or null.
void *kernel_for_i8(int L, int S, int GT, int NT, bool bim);
// The split-word instance (NS = 4, kernels_bits_split.cu) for a shape, or null.
void *kernel_for_split(int L, int S, int GT, int NT, bool bim);
bool bits_plan_fits(const BitsPlan &plan, int32_t R);
cudaError_t build_field4(const RealView &v, BitsPlan &plan, cudaStream_t st);
void free_bits_plan(BitsPlan &plan);
// n_sweeps sweeps; when exchange is true the launch ends with exchange step j (energies, swap
// decisions, permutation, measurement when j >= measure_from).
// With mh set (mh->mh > 0) the sweeps are multi-hit double-checkerboard sweeps.
// n_intervals > 1 (grid-wide plan with the exchange only): that many exchange intervals of n_sweeps
// sweeps each in one launch, exchange steps j, j + 1, ...
cudaError_t launch_sweeps_bits(const RealView &v, const BitsPlan &plan, uint32_t sweep0, int32_t n_sweeps,
                               bool exchange, uint32_t j, int64_t measure_from, double J, double h,
                               cudaStream_t st, const MultiHit *mh = nullptr, int32_t n_intervals = 1);

}  // namespace rfim
