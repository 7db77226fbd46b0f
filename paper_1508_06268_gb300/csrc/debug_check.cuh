// Bounds checks of the debug build.  With -DRFIM_DEBUG (the library flavour librfim_debug.so), a
// failed check records its bit in the launch's device error word and the caller replaces the
// offending index or address by a harmless one, so every thread still reaches every barrier and
// the kernel ends normally; the host reports the word as RFIM_EBOUNDS.  Nothing traps.  Without
// RFIM_DEBUG every check is the constant true and costs nothing.
#pragma once
#include <cstdint>

namespace rfim {

// Error-word bits (bits 0-7 are the bounded waits of the grid-wide plan).
constexpr unsigned kDbgLattice = 1u << 8;    // shared-memory lattice index outside the slab
constexpr unsigned kDbgTable = 1u << 9;      // decision-table slot outside dynamic shared memory
constexpr unsigned kDbgRank = 1u << 10;      // DSMEM peer rank outside the cluster
constexpr unsigned kDbgPartition = 1u << 11; // grid-wide partition: plane, piece or owner out of range
constexpr unsigned kDbgScratch = 1u << 12;   // no-alloc scratch slot beyond the static array
constexpr unsigned kDbgGlobal = 1u << 13;    // global lattice index outside the realization
constexpr unsigned kDbgMask = 0xFF00u;

#ifdef RFIM_DEBUG
constexpr bool kDebugBuild = true;
__device__ __forceinline__ bool dbg_check(unsigned *err, bool ok, unsigned bit) {
  if (!ok && err) atomicOr(err, bit);
  return ok;
}
__device__ __forceinline__ uint32_t dyn_smem_bytes() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_ctas() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
#define RFIM_DCHECK(err, cond, bit) ::rfim::dbg_check((err), (cond), (bit))
#else
constexpr bool kDebugBuild = false;
#define RFIM_DCHECK(err, cond, bit) true
#endif

}  // namespace rfim
