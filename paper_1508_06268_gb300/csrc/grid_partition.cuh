// Partition of a realization's (replica group, z plane) units over the CTAs of a cooperative
// launch, for the grid-wide bit-layout sweep (kernels_grid.cuh).  Host and device.
//
// Units u = g L + z for replica groups g = 0..NG-1 (of G replicas) and planes z = 0..L-1.  CTA k
// owns the contiguous units [a_k, a_{k+1}) with a_k = floor(k U / P), U = NG L, P CTAs; its range
// splits into "pieces" (maximal runs inside one group).  The z neighbours of a piece's first and
// last planes (periodic in z) belong to the CTAs owner(u) = floor(((u + 1) P - 1) / U).
#pragma once
#include <cstdint>

namespace rfim {

constexpr int kGridGroup = 4;      // default replicas per unit (processed together, one field load each)
constexpr int kGridMaxPieces = 4;  // pieces per CTA (checked on the host)

struct GridPart {
  int32_t L, NG, P;  // planes per replica, replica groups, CTAs
  int64_t U;         // units
};

__host__ __device__ __forceinline__ int64_t grid_begin(const GridPart &gp, int k) { return (int64_t)k * gp.U / gp.P; }

__host__ __device__ __forceinline__ int grid_owner(const GridPart &gp, int64_t u) {
  return (int)(((u + 1) * gp.P - 1) / gp.U);
}

struct Piece {
  int32_t g, z0, n;  // group, first plane, planes
  int32_t lu0;       // index of its first plane among the CTA's units
};

// Pieces of CTA k (returns their number).
__host__ __device__ __forceinline__ int grid_pieces(const GridPart &gp, int k, Piece out[kGridMaxPieces]) {
  const int64_t a = grid_begin(gp, k), b = grid_begin(gp, k + 1);
  int np = 0;
  for (int64_t u = a; u < b && np < kGridMaxPieces;) {
    const int32_t g = (int32_t)(u / gp.L), z = (int32_t)(u % gp.L);
    const int64_t end = b < (int64_t)(g + 1) * gp.L ? b : (int64_t)(g + 1) * gp.L;
    out[np].g = g;
    out[np].z0 = z;
    out[np].n = (int32_t)(end - u);
    out[np].lu0 = (int32_t)(u - a);
    ++np;
    u = end;
  }
  return np;
}

// Index of CTA k among the CTAs that own planes of group g (0 for the owner of plane 0).
__host__ __device__ __forceinline__ int grid_slab_of(const GridPart &gp, int k, int g) {
  return k - grid_owner(gp, (int64_t)g * gp.L);
}

}  // namespace rfim
