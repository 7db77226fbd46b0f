// Bit-layout (multi-spin coded) checkerboard sweep kernel, resident in shared memory, with the
// energy reduction and the exchange step fused into its tail.
//
// One cluster of S CTAs holds G replicas of a realization; CTA `rank` holds the z planes
// [rank L/S, (rank + 1) L/S) of both colours of all G replicas in shared memory for the whole
// launch and runs n sweeps (colour 0 half-sweep, colour 1 half-sweep; Eq. 3) before writing the
// lattices back.  Halo planes z0 - 1 and z0 + L/S come from the neighbouring CTAs of the cluster
// through distributed shared memory; a cluster barrier separates half-sweeps (S = 1: the CTA
// barrier).  A thread updates one 32-site word for GT replicas: neighbour counts by bit-sliced
// adders, then per Philox block (4 sites) one table lookup and one compare per site; the float
// field of those 4 sites is loaded once for all GT replicas.
//
// Exchange tail (optional): every CTA reduces the bond sum, magnetisation and field term of its
// slab of each of its replicas (Eq. 1) into per-slab partials; the last CTA of the grid to arrive
// (atomic arrival counter) adds the partials in slab order, forms E = -J B - F and takes the
// exchange step and the measurement (exchange.cuh).  No CTA waits for another.
#pragma once
#include <cstdint>

#include "bits_layout.cuh"
#include "debug_check.cuh"
#include "decide.cuh"
#include "exchange.cuh"
#include "internal.h"
#include "philox.cuh"

namespace rfim {

#ifndef RFIM_BLOCK_UNROLL
#define RFIM_BLOCK_UNROLL 8
#endif
// Unroll factor of the Philox-block loop of the sweep (compile-time experiment knob).
constexpr int kBlockUnroll = RFIM_BLOCK_UNROLL;

// Per-realization progress kept on the device by batched launches: the last work item of a
// realization advances it after the exchange step (sweep and exchange counters, intervals left).
struct SlotCtl {
  uint32_t sweep0;         // sweep index of the next interval
  uint32_t j;              // exchange step of the next interval
  int32_t intervals_left;  // 0: finished (its items are skipped)
  int32_t nsw;             // sweeps per interval
  int64_t measure_from;
  unsigned long long done_ns;  // device time stamp when intervals_left reached 0
};

// Arguments of the fused exchange tail.  Partials are [Rcap][S]; counter is zero between launches
// and `expected` arrivals (CTAs or work items) complete the realization.
// Fixed-point form of a float field for exact energy sums: H_i = rint(hh_i / 2^qe) with
// |H_i| < 2^39, so that H_i is five bytes (four unsigned, the top one signed); Htot = sum_i H_i.
struct FieldQuant {
  long long Htot;
  int qe;
  unsigned fmax;  // largest |hh_i| as float bits (while building)
};

struct ExchArgs {
  int32_t enabled;
  uint32_t j;
  int64_t measure_from;
  double J, h;
  long long *partB, *partM, *partFi;
  double *partF;
  unsigned int *counter;
  unsigned int expected;
  SlotCtl *ctl;       // batched launches only (else null)
  unsigned int *err;  // error word: bit 0 = a bounded device wait expired
  // structure factor of the correlation length (batched launches that measure it; else null):
  // cos / sin(K t) tables [L], per-replica F of this interval [R], sums per temperature [R]
  const double *kcos, *ksin;
  double *Fr, *sumF;
  // fixed-point field of the energy tail (both null: error-free float sums of hh instead):
  // H = rint(hh / q), q = 2^qe, as byte limbs (flimb_index) and the lattice sum of H
  const uint4 *flimb;
  const FieldQuant *fquant;
};

__host__ __device__ __forceinline__ int64_t field4_index(int c, int64_t wq, int j, int64_t wpad) {
  return ((int64_t)c * wpad + (wq & ~31LL)) * 8 + (int64_t)j * 32 + (wq & 31);
}

// uint4 s of colour c, word wq: s < 8, limbs 0..3 (.x .. .w) of the four sites 4s + k (byte k);
// s = 8, 9: limb 4 of blocks 4(s - 8) .. 4(s - 8) + 3 (.x .. .w), each byte one site.  Words are
// the fastest index, so a warp's loads of one s are contiguous.
__host__ __device__ __forceinline__ int64_t flimb_index(int c, int64_t wq, int s, int64_t wpad) {
  return ((int64_t)c * 10 + s) * wpad + wq;
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t dsmem_load(const uint32_t *local, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
  uint32_t ra, val;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(val) : "r"(ra) : "memory");
  return val;
}

template <int S>
__device__ __forceinline__ void sync_slabs() {
  if (S == 1) {
    __syncthreads();
  } else {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
}

// Per-site table offsets from bit slices.  For Philox block j (bits j of the four bytes) the
// table offset of site k is bits 3..6 (float field: up-count c0 c1 c2, spin) or 2..6 (bimodal:
// plus field bit) of byte k.  The slices are pair-interleaved once per word so that each block
// needs one mux and one rotate (two for bimodal) instead of a shift and mask per slice.
struct PairSlices {
  uint32_t pa, qa, pb, qb;  // (c0,c1) and (c2,s) for even / odd blocks, (c2,s) pre-rotated by 2
  uint32_t f3, f4;          // bimodal field bits rotated for odd / even blocks
};

__device__ __forceinline__ uint32_t rotl(uint32_t x, int n) { return __funnelshift_l(x, x, n); }
__device__ __forceinline__ uint32_t rotr(uint32_t x, int n) { return __funnelshift_r(x, x, n); }
__device__ __forceinline__ uint32_t mux(uint32_t a, uint32_t b, uint32_t m) { return (a & m) | (b & ~m); }

__device__ __forceinline__ PairSlices make_pairs(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t s, uint32_t f) {
  PairSlices r;
  r.pa = mux(c0, c1 << 1, 0x55555555u);
  r.qa = mux(c0 >> 1, c1, 0x55555555u);
  r.pb = rotl(mux(c2, s << 1, 0x55555555u), 2);
  r.qb = rotl(mux(c2 >> 1, s, 0x55555555u), 2);
  r.f4 = rotl(f, 4);
  r.f3 = rotl(f, 3);
  return r;
}

// j is a compile-time constant once the block loop is unrolled.
template <bool BIM>
__device__ __forceinline__ uint32_t block_offsets(const PairSlices &p, int j) {
  const int m = j >> 1;
  const uint32_t a = (j & 1) ? p.qa : p.pa;
  const uint32_t b = (j & 1) ? p.qb : p.pb;
  const uint32_t ma = 0x03030303u << (2 * m);  // (c0, c1) at bits 2m, 2m+1 of every byte
  uint32_t z = mux(a, b, ma);                   // (c2, s) at 2m+2, 2m+3 (cyclic)
  if (BIM) {
    const uint32_t f = (j & 1) ? p.f3 : p.f4;   // field bit at 2m+4 (cyclic)
    z = mux(f, z, rotl(0x01010101u, (2 * m + 4) & 31));
    return rotr(z, (2 * m - 2) & 31) & 0x7C7C7C7Cu;  // bit 2m -> bit 2 of every byte
  }
  return rotr(z, (2 * m - 3) & 31) & 0x78787878u;    // bit 2m -> bit 3 of every byte
}

// ---- per-replica decision tables in shared memory ------------------------------------------
// A replica's table (bimodal: 32 thresholds - 1, indexed by up-count, spin, field bit; float
// field: 16 pairs (fl(b J n), b), b = fl(-2 beta log2 e) signed by the spin, indexed by up-count
// and spin) sits in its own 256-byte slot aligned to 256 bytes.  Byte k of a block's
// offset word then holds site k's byte offset within the slot, and one byte permute with the
// slot address forms the entry address.
constexpr uint32_t kTabSlot = 256;

// Dynamic shared-memory bytes for n tables, with the alignment slack.
__host__ __device__ constexpr size_t tab_bytes(int n) { return (size_t)(n + 1) * kTabSlot; }

// Shared-window address of the first slot at or after p.
__device__ __forceinline__ uint32_t tab_slot0(const void *p) {
  return ((uint32_t)__cvta_generic_to_shared(p) + kTabSlot - 1u) & ~(kTabSlot - 1u);
}

// Fills the tables of n slots, slot g for temperature temp_of(g), with all threads of the CTA.
// `base` is any generic pointer into dynamic shared memory at or before the slots.
template <bool BIM, class F>
__device__ __forceinline__ void tab_fill_temps(const RealView &v, void *base, uint32_t slot0, int n, F temp_of) {
  constexpr int E = BIM ? 32 : 16;
  char *gen = reinterpret_cast<char *>(base) + (slot0 - (uint32_t)__cvta_generic_to_shared(base));
  for (int t = threadIdx.x; t < n * E; t += blockDim.x) {
    const int g = t / E, i = t % E;
    const int k = temp_of(g);
    char *slot = gen + (size_t)g * kTabSlot;
    if (BIM) {
      reinterpret_cast<uint32_t *>(slot)[i] = v.thr[(int64_t)k * 32 + i];
    } else {
      const float b = (i >> 3) ? v.b2l[k] : -v.b2l[k];
      reinterpret_cast<float2 *>(slot)[i] = make_float2(__fmul_rn(b, v.gjn[i & 7]), b);
    }
  }
}

// The same with slot g for the temperature of replica replica_of(g).
template <bool BIM, class F>
__device__ __forceinline__ void tab_fill(const RealView &v, void *base, uint32_t slot0, int n, F replica_of) {
  tab_fill_temps<BIM>(v, base, slot0, n, [&](int g) { return v.r2t[replica_of(g)]; });
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t r;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r) : "r"(a));
  return r;
}

__device__ __forceinline__ float2 lds_f2(uint32_t a) {
  float2 r;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(a));
  return r;
}

// Decisions of Philox block j of one word of one replica: sites 4j + k (k = 0..3) at bits 8k + j,
// table slot `slot`, float field h4 of those sites.  Bimodal: accepted sites set their bit of
// `flip`; float field: the acceptance sign bits are shifted into fk[k] (blocks visited j = 7..0,
// so block j ends at bit j of fk[k]).
template <bool BIM>
__device__ __forceinline__ void decide_block(const Words4 &w, const PairSlices &ps, int j, uint32_t slot,
                                             const float4 &h4, uint32_t &flip, uint32_t (&fk)[4]) {
  const uint32_t offs = block_offsets<BIM>(ps, j);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t a = __byte_perm(offs, slot, 0x7650u | (uint32_t)k);
    if (BIM) {
      if (accept_table(w.w[k], lds_u32(a))) flip |= 1u << (8 * k + j);
    } else {
      const float hk = k == 0 ? h4.x : k == 1 ? h4.y : k == 2 ? h4.z : h4.w;
      const float2 e = lds_f2(a);
      fk[k] = __funnelshift_l(accept_float_sign(w.w[k], e.x, hk, e.y), fk[k], 1);
    }
  }
}

// The six other-colour neighbour words of local word (zl, iw) from plane array O (this CTA's
// planes; halo planes from the neighbouring ranks).
template <int L, int S>
__device__ __forceinline__ void neighbour_words(const uint32_t *O, int zl, int iw, uint32_t p0, int up_rank,
                                                int dn_rank, uint32_t nb[6]) {
  constexpr int P = BitsGeom<L>::P, PZ = L / S;
  const uint32_t same = O[zl * P + iw];
  const uint32_t next = O[zl * P + (iw + 1) % P];
  const uint32_t prev = O[zl * P + (iw + P - 1) % P];
  nb_xy<L>(same, next, prev, p0, nb[0], nb[1], nb[2], nb[3]);
  if (zl + 1 < PZ)
    nb[4] = O[(zl + 1) * P + iw];
  else
    nb[4] = S == 1 ? O[iw] : dsmem_load(O + iw, up_rank);
  if (zl > 0)
    nb[5] = O[(zl - 1) * P + iw];
  else
    nb[5] = S == 1 ? O[(PZ - 1) * P + iw] : dsmem_load(O + (PZ - 1) * P + iw, dn_rank);
}

// Replicas reduced together by the fused exchange tail.  Every L = 32 launch shape holds at most
// two replicas per CTA, and there, with a float field, the four-replica tail's registers slowed
// the sweeps themselves (L = 32, R = 70: 49.8 -> 55.5 us per 10 sweeps), so that case reduces
// one replica at a time (with the bimodal field four stays faster: 53.4 against 56.9 us per
// interval).
constexpr int kTailRB = 4;
template <int L, bool BIM>
constexpr int tail_rb() { return (L == 32 && !BIM) ? 1 : kTailRB; }

template <typename T>
__device__ __forceinline__ T warp_reduce_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Shared-memory marginals of the fused structure-factor measurement: 3 L ints per replica.
constexpr int kXiMargInts = 768;
__device__ __forceinline__ int *xi_marg_smem() {
  __shared__ int m[kXiMargInts];
  return m;
}

// Structure factor F of the correlation length (Sec. 7; the spins s_i read for the printed h_i)
// of replicas [r0, r0 + gact), whole lattices in shared memory (one slab per replica):
// F = (1 / 3N) sum over the axes d of |sum_t S_d[t] e^{i K t}|^2, K = 2 pi / L, from the exact
// integer marginals S_d[t] (sum of the spins with coordinate t along axis d).  Word wq of colour
// c holds sites q = 32 wq + i (in-word site i at bit 8 (i & 3) + (i >> 2)), i.e. RW = 32 / (L/2)
// rows (y, z) of L/2 sites each, row rr at y = y0 + rr, x = 2 (i mod L/2) + ((c + y + z) & 1).
// y and z marginals come from popcounts of rows and words; for x a warp takes 32 words and, per
// in-word site i, ballots the spins and the row parities, counted by lane i.  The Fourier sums run
// in double, one warp per replica with a fixed shuffle tree; F of replica r0 + g goes to xa.Fr.
template <int L>
__device__ __forceinline__ void xi_replicas(const uint32_t *sp, int r0, int gact, const ExchArgs &xa, int32_t N) {
  constexpr int W = BitsGeom<L>::W, P = BitsGeom<L>::P, Lh = L / 2, RW = 32 / Lh, NB = (W + 31) / 32;
  constexpr int CH = kXiMargInts / (3 * L);
  constexpr uint32_t kRowMask = ((1u << (Lh / 4)) - 1u) * 0x01010101u;
  static_assert(L >= 8 && L <= 64 && CH >= 1, "rows of one colour must tile a word");
  int *marg = xi_marg_smem();
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int g0 = 0; g0 < gact; g0 += CH) {
    const int ng = min(CH, gact - g0);
    for (int t = tid; t < ng * 3 * L; t += nt) marg[t] = 0;
    __syncthreads();
    for (int u = wid; u < ng * 2 * NB; u += nw) {
      const int gl = u / (2 * NB), c = (u / NB) & 1, wq = (u % NB) * 32 + lane;
      const bool valid = wq < W;
      const uint32_t w = valid ? sp[((size_t)(g0 + gl) * 2 + c) * W + wq] : 0u;
      int *mg = marg + gl * 3 * L;
      const int row0 = wq * RW, z = row0 / L, y0 = row0 % L;
      if (valid) {
#pragma unroll
        for (int rr = 0; rr < RW; ++rr) atomicAdd(&mg[L + y0 + rr], 2 * __popc(w & (kRowMask << (rr * (Lh / 4)))) - Lh);
      }
      if (P >= 32) {  // the warp's 32 words share one plane
        int zs = 2 * __popc(w) - 32;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) zs += __shfl_xor_sync(0xffffffffu, zs, o);
        if (lane == 0) atomicAdd(&mg[2 * L + z], zs);
      } else if (valid) {
        atomicAdd(&mg[2 * L + z], 2 * __popc(w) - 32);
      }
      const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
      const uint32_t odd0 = __ballot_sync(0xffffffffu, valid && ((c + y0 + z) & 1));
      int ax0 = 0, ax1 = 0;  // columns x = 2 (lane mod L/2) and that + 1
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const uint32_t m = __ballot_sync(0xffffffffu, (w >> (8 * (i & 3) + (i >> 2))) & 1u);
        if (lane == i) {
          const uint32_t odd = ((i / Lh) & 1) ? (vmask & ~odd0) : odd0, even = vmask & ~odd;
          ax0 = 2 * __popc(m & even) - __popc(even);
          ax1 = 2 * __popc(m & odd) - __popc(odd);
        }
      }
      atomicAdd(&mg[2 * (lane % Lh)], ax0);
      atomicAdd(&mg[2 * (lane % Lh) + 1], ax1);
    }
    __syncthreads();
    for (int gl = wid; gl < ng; gl += nw) {
      const int *mg = marg + gl * 3 * L;
      double F = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double cs = 0.0, sn = 0.0;
        for (int t = lane; t < L; t += 32) {
          cs = __dadd_rn(cs, __dmul_rn(xa.kcos[t], (double)mg[d * L + t]));
          sn = __dadd_rn(sn, __dmul_rn(xa.ksin[t], (double)mg[d * L + t]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          cs = __dadd_rn(cs, __shfl_down_sync(0xffffffffu, cs, o));
          sn = __dadd_rn(sn, __shfl_down_sync(0xffffffffu, sn, o));
        }
        F = __dadd_rn(F, __dadd_rn(__dmul_rn(cs, cs), __dmul_rn(sn, sn)));
      }
      if (lane == 0) {
        xa.Fr[r0 + g0 + gl] = F / (3.0 * (double)N);
        __threadfence();
      }
    }
    __syncthreads();
  }
}

// Fused exchange tail of an interval (Eq. 1 energies, then the last arrival takes exchange step
// xa.j): slab partials of each replica from the lattice still in shared memory, an arrival count,
// and for the last arrival the ordered reduction, E = -J B - F, exchange and measurement.  XI
// (whole replicas, S = 1): on measuring steps with xa.sumF set, also the structure factor.
template <int L, int S, bool BIM, bool XI = false, int RB = tail_rb<L, BIM>()>
__device__ __forceinline__ void interval_tail(const RealView &v, int G, int r0, int gact, int rank, int nsw,
                                              const float4 *__restrict__ field4, const ExchArgs &xa) {
  using Gm = BitsGeom<L>;
  constexpr int P = Gm::P, W = Gm::W, PZ = L / S, WC = PZ * P;
  constexpr int64_t WPAD = (W + 31) / 32 * 32;
  extern __shared__ __align__(16) uint32_t sm[];
  const int up_rank = (rank + 1) % S, dn_rank = (rank + S - 1) % S;
  const int z0 = rank * PZ;
  const uint32_t *sp = sm;
  const int nt = blockDim.x, tid = threadIdx.x;

  // ---- energy partials of this slab (Eq. 1): B over colour-0 words x their six neighbour words,
  // M over all words and the field term per thread, up to RB replicas at a time (each word's field
  // is loaded once for all of them; one barrier pair reduces them all: warp trees, then one warp
  // per replica over the warps).  Field term: bimodal, the exact integer sum of hb s; float field
  // with the fixed-point limbs (xa.flimb), the exact integer sum of H over the up spins of the
  // slab, H = rint(hh / q) in five byte limbs summed by four-way byte dot products against the
  // spin bits of each Philox block (F = q (2 sum_up H - sum_all H) in the last CTA); without them,
  // an error-free float sum (Sum2).
  __shared__ int red_i[BIM ? 3 : 2][RB][32];
  __shared__ long long red_l[BIM ? 1 : RB][32];
  __shared__ double red_d[RB][32];
  __shared__ int last_cta;
  const int lane = tid & 31, wid = tid >> 5, nw = (nt + 31) >> 5;
  const bool limbs = !BIM && xa.flimb != nullptr;
  for (int g0 = 0; g0 < gact; g0 += RB) {
    const int ng = min(RB, gact - g0);
    int b[RB], m[RB], fi[RB], hs[RB];
    unsigned hu[RB][4];
    float fs[RB], fe[RB];
#pragma unroll
    for (int gg = 0; gg < RB; ++gg) {
      b[gg] = m[gg] = fi[gg] = hs[gg] = 0;
      fs[gg] = fe[gg] = 0.f;
#pragma unroll
      for (int l = 0; l < 4; ++l) hu[gg][l] = 0u;
    }
    for (int t = tid; t < 2 * WC; t += nt) {
      const int c = t / WC, wl = t % WC;
      const int zl = wl / P, iw = wl % P, z = z0 + zl;
      const int64_t wq = (int64_t)z * P + iw;
      const uint32_t hb = BIM ? v.hbits[(int64_t)c * W + wq] : 0u;
      uint32_t self[RB];
#pragma unroll
      for (int gg = 0; gg < RB; ++gg) {
        self[gg] = gg < ng ? sp[((size_t)(g0 + gg) * 2 + c) * WC + wl] : 0u;
        if (gg >= ng) continue;
        m[gg] += 2 * __popc(self[gg]) - 32;
        if (c == 0) {
          uint32_t nb[6];
          neighbour_words<L, S>(sp + ((size_t)(g0 + gg) * 2 + 1) * WC, zl, iw, parity0_mask<L>(0, z, iw), up_rank,
                                dn_rank, nb);
#pragma unroll
          for (int d = 0; d < 6; ++d) b[gg] += 32 - 2 * __popc(self[gg] ^ nb[d]);
        }
        if (BIM) fi[gg] += 32 - 2 * __popc(self[gg] ^ hb);
      }
      if (limbs) {
        // block j: byte k of (self >> j) & 0x01010101 is the up bit of site 4j + k
        const uint4 top0 = __ldg(xa.flimb + flimb_index(c, wq, 8, WPAD));
        const uint4 top1 = __ldg(xa.flimb + flimb_index(c, wq, 9, WPAD));
        const uint32_t top[8] = {top0.x, top0.y, top0.z, top0.w, top1.x, top1.y, top1.z, top1.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint4 lo = __ldg(xa.flimb + flimb_index(c, wq, j, WPAD));
#pragma unroll
          for (int gg = 0; gg < RB; ++gg) {
            if (gg >= ng) continue;
            const uint32_t up = (self[gg] >> j) & 0x01010101u;
            hu[gg][0] = __dp4a(up, lo.x, hu[gg][0]);
            hu[gg][1] = __dp4a(up, lo.y, hu[gg][1]);
            hu[gg][2] = __dp4a(up, lo.z, hu[gg][2]);
            hu[gg][3] = __dp4a(up, lo.w, hu[gg][3]);
            hs[gg] = __dp4a((int)up, (int)top[j], hs[gg]);  // top limb signed, up bytes 0 or 1
          }
        }
      } else if (!BIM) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 q4 = __ldg(field4 + field4_index(c, wq, j, WPAD));
          const float hk[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
          for (int gg = 0; gg < RB; ++gg) {
            if (gg >= ng) continue;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float term = ((self[gg] >> (8 * k + j)) & 1u) ? hk[k] : -hk[k];
              const float tsum = __fadd_rn(fs[gg], term);
              const float bp = __fsub_rn(tsum, fs[gg]);
              fe[gg] = __fadd_rn(fe[gg], __fadd_rn(__fsub_rn(fs[gg], __fsub_rn(tsum, bp)), __fsub_rn(term, bp)));
              fs[gg] = tsum;
            }
          }
        }
      }
    }
#pragma unroll
    for (int gg = 0; gg < RB; ++gg) {
      const int tb = warp_reduce_sum(b[gg]), tm = warp_reduce_sum(m[gg]);
      // field integer: bimodal sum of hb s (int), or the up-spin sum of H from its limbs
      if constexpr (BIM) {
        const int tf = warp_reduce_sum(fi[gg]);
        if (lane == 0) red_i[2][gg][wid] = tf;
      } else {
        long long fl = 0;
        if (limbs)
          fl = (long long)hu[gg][0] + ((long long)hu[gg][1] << 8) + ((long long)hu[gg][2] << 16) +
               ((long long)hu[gg][3] << 24) + ((long long)hs[gg] << 32);
        const long long tf = warp_reduce_sum(fl);
        if (lane == 0) red_l[gg][wid] = tf;
      }
      const double td = (BIM || limbs) ? 0.0 : warp_reduce_sum((double)fs[gg] + (double)fe[gg]);
      if (lane == 0) {
        red_i[0][gg][wid] = tb;
        red_i[1][gg][wid] = tm;
        red_d[gg][wid] = td;
      }
    }
    __syncthreads();
    if (wid < ng) {  // warp gg adds the warps' partials of replica g0 + gg
      const int gg = wid;
      const long long tb = warp_reduce_sum(lane < nw ? (long long)red_i[0][gg][lane] : 0LL);
      const long long tm = warp_reduce_sum(lane < nw ? (long long)red_i[1][gg][lane] : 0LL);
      const long long tf =
          warp_reduce_sum(lane < nw ? (BIM ? (long long)red_i[BIM ? 2 : 0][gg][lane] : red_l[BIM ? 0 : gg][lane]) : 0LL);
      const double td = warp_reduce_sum(lane < nw ? red_d[gg][lane] : 0.0);
      if (lane == 0) {
        const int64_t slot = (int64_t)(r0 + g0 + gg) * S + rank;
        xa.partB[slot] = tb;
        xa.partM[slot] = tm;
        xa.partFi[slot] = tf;
        xa.partF[slot] = td;
      }
    }
    __syncthreads();
  }
  if constexpr (XI && S == 1) {
    if (xa.sumF && (int64_t)xa.j >= xa.measure_from) xi_replicas<L>(sp, r0, gact, xa, v.N);
  }
  sync_slabs<S>();  // peers may still read this CTA's halo planes
  if (tid == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(xa.counter, 1u);
    last_cta = prev == xa.expected - 1;
  }
  __syncthreads();
  if (!last_cta) return;
  __threadfence();
  for (int r = tid; r < v.R; r += nt) {
    long long tb = 0, tm = 0, tf = 0;
    double td = 0.0;
    for (int q = 0; q < S; ++q) {
      const int64_t slot = (int64_t)r * S + q;
      tb += __ldcg(xa.partB + slot);
      tm += __ldcg(xa.partM + slot);
      tf += __ldcg(xa.partFi + slot);
      td += __ldcg(xa.partF + slot);
    }
    const double F = BIM ? xa.h * (double)tf
                         : (xa.flimb ? ldexp((double)(2 * tf - xa.fquant->Htot), xa.fquant->qe) : td);
    v.E[r] = -xa.J * (double)tb - F;
    v.M[r] = tm;
  }
  __syncthreads();
  if constexpr (XI && S == 1)
    exchange_and_measure(v, xa.j, xa.measure_from, xa.Fr, xa.sumF);
  else
    exchange_and_measure(v, xa.j, xa.measure_from);
  if (tid == 0) {
    *xa.counter = 0u;
    if (xa.ctl) {
      SlotCtl *c = xa.ctl;
      c->sweep0 += (uint32_t)nsw;
      c->j += 1u;
      c->intervals_left -= 1;
      if (c->intervals_left == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        c->done_ns = t;
      }
      __threadfence();
    }
  }
  __syncthreads();
}


// Per byte, bit b of the low nibble moves to the b-th set bit of PAT (four set bits).
template <uint32_t PAT>
__device__ __forceinline__ uint32_t deposit_nibbles(uint32_t x) {
  uint32_t out = 0u;
  int b = 0;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    if ((PAT >> p) & 1u) {
      const uint32_t moved = p >= b ? x << (p - b) : x >> (b - p);
      out |= moved & (0x01010101u << p);
      ++b;
    }
  }
  return out;
}

// Metropolis update of one word (32 sites of colour c at plane zl, word iw of the slab) in the GT
// replicas of group grp: neighbour counts from the other colour's words, one Philox block per
// (block j, replica) with counter (8 wq + j, r, ctr2, tag), decisions, and the flipped words
// written back.  Only the blocks with their bit set in PAT are updated (0xFF: all; otherwise four
// of them, whose float-field sign bits are collected side by side and then moved to their bytes'
// bit j).  Replicas past the end of a partial group repeat the last one; only their write is
// skipped.
template <int L, int S, int GT, bool BIM, uint32_t PAT>
__device__ __forceinline__ void update_word(const RealView &v, uint32_t *sp, int c, int zl, int iw, int z0, int grp,
                                            int gact, int r0, uint32_t ctr2, uint32_t tag, uint32_t slot0,
                                            const float4 *__restrict__ field4, int up_rank, int dn_rank) {
  static_assert(PAT == 0xFFu || __builtin_popcount(PAT) == 4, "a pass updates all blocks or four of them");
  using Gm = BitsGeom<L>;
  constexpr int P = Gm::P, W = Gm::W, PZ = L / S, WC = PZ * P;
  constexpr int64_t WPAD = (W + 31) / 32 * 32;
  const int wl = zl * P + iw, z = z0 + zl;
  const int64_t wq = (int64_t)z * P + iw;
  float4 hh4[8] = {};
  if (!BIM) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if ((PAT >> j) & 1u) hh4[j] = __ldg(field4 + field4_index(c, wq, j, WPAD));
  }
  const uint32_t p0 = parity0_mask<L>(c, z, iw);
  uint32_t c0[GT], c1[GT], c2[GT], sf[GT], flip[GT];
#pragma unroll
  for (int gg = 0; gg < GT; ++gg) {
    const int g = min(grp * GT + gg, gact - 1);
    uint32_t nb[6];
    neighbour_words<L, S>(sp + ((size_t)g * 2 + (c ^ 1)) * WC, zl, iw, p0, up_rank, dn_rank, nb);
    count6(nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], c0[gg], c1[gg], c2[gg]);
    sf[gg] = sp[((size_t)g * 2 + c) * WC + wl];
    flip[gg] = 0u;
  }
  const uint32_t fb = BIM ? v.hbits[(int64_t)c * W + wq] : 0u;
  PairSlices ps[GT];
#pragma unroll
  for (int gg = 0; gg < GT; ++gg) ps[gg] = make_pairs(c0[gg], c1[gg], c2[gg], sf[gg], fb);
  // float field: flip = fk[k] << 8k once all blocks are done
  uint32_t fk[GT][4];
#pragma unroll
  for (int gg = 0; gg < GT; ++gg)
#pragma unroll
    for (int k = 0; k < 4; ++k) fk[gg][k] = 0u;
#pragma unroll kBlockUnroll
  for (int jj = 0; jj < 8; ++jj) {
    const int j = 7 - jj;
    if ((PAT >> j) & 1u) {
#pragma unroll
      for (int gg = 0; gg < GT; ++gg) {
        const int g = min(grp * GT + gg, gact - 1);
        const Words4 w = philox10(v.seed, v.realization, (uint32_t)(8 * wq + j), (uint32_t)(r0 + g), ctr2, tag);
        decide_block<BIM>(w, ps[gg], j, slot0 + (uint32_t)g * kTabSlot, hh4[j], flip[gg], fk[gg]);
      }
    }
  }
  if (!BIM) {
#pragma unroll
    for (int gg = 0; gg < GT; ++gg) {
      flip[gg] = fk[gg][0] | (fk[gg][1] << 8) | (fk[gg][2] << 16) | (fk[gg][3] << 24);
      if (PAT != 0xFFu) flip[gg] = deposit_nibbles<PAT>(flip[gg]);
    }
  }
#pragma unroll
  for (int gg = 0; gg < GT; ++gg) {
    const int g = grp * GT + gg;
    if (GT > 1 && g >= gact) continue;
    sp[((size_t)g * 2 + c) * WC + wl] = sf[gg] ^ flip[gg];
  }
}

// int8 layout staged as bits: the 32 sites q = 32 wq + p (p = 4j + k) of a bit-layout word are
// the 32 consecutive 0/1 bytes at spins8 + 32 wq of the same colour; byte 4j + k goes to bit 8k + j,
// i.e. the word is the OR of the eight 4-byte groups shifted by j.
__device__ __forceinline__ uint32_t pack_int8_word(const uint8_t *p32) {
  const uint4 a = *reinterpret_cast<const uint4 *>(p32), b = *reinterpret_cast<const uint4 *>(p32 + 16);
  return a.x | (a.y << 1) | (a.z << 2) | (a.w << 3) | (b.x << 4) | (b.y << 5) | (b.z << 6) | (b.w << 7);
}
__device__ __forceinline__ void unpack_int8_word(uint32_t w, uint8_t *p32) {
  const uint32_t m = 0x01010101u;
  *reinterpret_cast<uint4 *>(p32) = make_uint4(w & m, (w >> 1) & m, (w >> 2) & m, (w >> 3) & m);
  *reinterpret_cast<uint4 *>(p32 + 16) = make_uint4((w >> 4) & m, (w >> 5) & m, (w >> 6) & m, (w >> 7) & m);
}

// Copies the slab (both colours) of replicas [r0, r0 + gact) between global and shared memory.
template <int L, int S, bool TO_SHARED>
__device__ __forceinline__ void copy_slab(const RealView &v, uint32_t *sp, int r0, int gact, int z0) {
  using Gm = BitsGeom<L>;
  constexpr int P = Gm::P, W = Gm::W, WC = (L / S) * P;
  for (int t = threadIdx.x; t < gact * 2 * WC; t += blockDim.x) {
    const int g = t / (2 * WC), rem = t % (2 * WC), c = rem / WC, wl = rem % WC;
    uint32_t *gw = v.bits + ((int64_t)(r0 + g) * 2 + c) * W + (int64_t)z0 * P + wl;
    if (TO_SHARED)
      sp[t] = *gw;
    else
      *gw = sp[t];
  }
}

// Block pair BG (blocks 2 BG and 2 BG + 1) of word wl of replica g (one replica per unit): the
// counts of the whole word, two Philox blocks and their decisions, and the flips xored into the
// word in shared memory.  The four block pairs of a word are run by four warps; they flip disjoint
// bits, and a pair's decisions read only its own bits of the word, so the order of their xors
// does not matter.
template <int L, int S, bool BIM, int BG>
__device__ __forceinline__ void split_unit(const RealView &v, uint32_t *sp, int c, int g, int wl, int z0, int r0,
                                           uint32_t sweep, uint32_t tag, uint32_t slot, const float4 *__restrict__ field4,
                                           int up_rank, int dn_rank) {
  using Gm = BitsGeom<L>;
  constexpr int P = Gm::P, W = Gm::W, PZ = L / S, WC = PZ * P;
  constexpr int64_t WPAD = (W + 31) / 32 * 32;
  const int zl = wl / P, iw = wl % P, z = z0 + zl;
  const int64_t wq = (int64_t)z * P + iw;
  float4 h[2] = {};
  if (!BIM) {
    h[0] = __ldg(field4 + field4_index(c, wq, 2 * BG, WPAD));
    h[1] = __ldg(field4 + field4_index(c, wq, 2 * BG + 1, WPAD));
  }
  uint32_t nb[6], c0, c1, c2;
  neighbour_words<L, S>(sp + ((size_t)g * 2 + (c ^ 1)) * WC, zl, iw, parity0_mask<L>(c, z, iw), up_rank, dn_rank, nb);
  count6(nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], c0, c1, c2);
  uint32_t *self = sp + ((size_t)g * 2 + c) * WC + wl;
  const uint32_t fb = BIM ? v.hbits[(int64_t)c * W + wq] : 0u;
  const PairSlices ps = make_pairs(c0, c1, c2, *self, fb);
  uint32_t flip = 0u, fk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int jj = 0; jj < 2; ++jj) {  // block 2 BG + 1, then 2 BG: the sign collectors end with block 2 BG at bit 0
    const int j = 2 * BG + 1 - jj;
    const Words4 w = philox10(v.seed, v.realization, (uint32_t)(8 * wq + j), (uint32_t)(r0 + g), sweep, tag);
    decide_block<BIM>(w, ps, j, slot, h[1 - jj], flip, fk);
  }
  if (!BIM) flip = (fk[0] | (fk[1] << 8) | (fk[2] << 16) | (fk[3] << 24)) << (2 * BG);
  atomicXor(self, flip);
}

// One exchange interval of replicas [r0, r0 + gact) of realization v, slab `rank` of S: load into
// shared memory, nsw sweeps, write back, and (xa.enabled) the energy partials and the exchange
// tail.  All threads of the CTA call it; blockDim.x threads, dynamic shared memory >= the plan's.
// I8: the realization is stored in the int8 layout (v.spins8) and staged here as bits: the slab is
// packed into shared memory on entry and unpacked back on exit (a word is 32 consecutive bytes).
// NS = 4 (with GT = 1): every word is updated by four warps, one block pair each (split_unit), so
// that small lattices, whose half-sweeps are too short to fill the SMs, run four times as many
// threads with a quarter of the Philox work each.
template <int L, int S, int GT, bool BIM, bool XI = false, bool I8 = false, int NS = 1>
__device__ __forceinline__ void bits_interval(const RealView &v, int G, int r0, int gact, int rank, uint32_t sweep0,
                                              int nsw, const float4 *__restrict__ field4, const ExchArgs &xa) {
  using Gm = BitsGeom<L>;
  constexpr int P = Gm::P, W = Gm::W, PZ = L / S, WC = PZ * P;
  constexpr int64_t WPAD = (W + 31) / 32 * 32;
  extern __shared__ __align__(16) uint32_t sm[];
  const int up_rank = (rank + 1) % S, dn_rank = (rank + S - 1) % S;
  const int z0 = rank * PZ;
  __syncthreads();  // a CTA may run several intervals back to back: shared memory is reused
  uint32_t *sp = sm;                        // [G][2][WC]
  uint32_t *tab = sm + (size_t)G * 2 * WC;  // G decision-table slots
  const uint32_t slot0 = tab_slot0(tab);
  const int nt = blockDim.x, tid = threadIdx.x;

  // debug build: the replica range, the decision-table slots and the cluster peers must lie
  // inside the realization, the dynamic shared memory and the cluster; otherwise nothing is
  // updated (every thread agrees, so the barriers still match)
  const bool ok = RFIM_DCHECK(xa.err, gact >= 1 && gact <= G && r0 >= 0 && r0 + gact <= v.R, kDbgGlobal) &&
                  RFIM_DCHECK(xa.err, slot0 + (uint32_t)gact * kTabSlot <= (uint32_t)__cvta_generic_to_shared(sm) + dyn_smem_bytes() &&
                                          (uint32_t)__cvta_generic_to_shared(tab) + kTabSlot - 1u >= slot0,
                              kDbgTable) &&
                  RFIM_DCHECK(xa.err, S == 1 || (cluster_ctas() == (uint32_t)S && up_rank < S && dn_rank < S), kDbgRank);
  for (int t = tid; ok && t < gact * 2 * WC; t += nt) {
    const int g = t / (2 * WC), rem = t % (2 * WC), c = rem / WC, wl = rem % WC;
    const int64_t gw = ((int64_t)(r0 + g) * 2 + c) * W + (int64_t)z0 * P + wl;
    sp[t] = I8 ? pack_int8_word(v.spins8 + 32 * gw) : v.bits[gw];
  }
  if (ok) tab_fill<BIM>(v, tab, slot0, gact, [&](int g) { return r0 + g; });
  sync_slabs<S>();

  const int ngroups = (gact + GT - 1) / GT;
  const int items = WC * ngroups;
  for (int s = 0; s < nsw; ++s) {
    const uint32_t sweep = sweep0 + (uint32_t)s;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const uint32_t tag = tag_word(kTagMetro, v.stage, (uint32_t)c);
      // the word update is written out here rather than called through update_word (which the
      // multi-hit kernel uses): the call changes the register allocation of this kernel (100 ->
      // 128 registers with spills for the float field at L = 64)
      if constexpr (NS == 4) {
        static_assert(GT == 1, "split words: one replica per unit");
        const int warp = tid >> 5, bg = warp & 3, quads = nt >> 7;
#pragma unroll 1
        for (int item = (warp >> 2) * 32 + (tid & 31); ok && item < items; item += quads * 32) {
          const int wl = item % WC, g = item / WC;
          if (!RFIM_DCHECK(xa.err, g < gact && wl < WC, kDbgLattice)) continue;
          const uint32_t slot = slot0 + (uint32_t)g * kTabSlot;
          switch (bg) {  // warp-uniform
            case 0: split_unit<L, S, BIM, 0>(v, sp, c, g, wl, z0, r0, sweep, tag, slot, field4, up_rank, dn_rank); break;
            case 1: split_unit<L, S, BIM, 1>(v, sp, c, g, wl, z0, r0, sweep, tag, slot, field4, up_rank, dn_rank); break;
            case 2: split_unit<L, S, BIM, 2>(v, sp, c, g, wl, z0, r0, sweep, tag, slot, field4, up_rank, dn_rank); break;
            default: split_unit<L, S, BIM, 3>(v, sp, c, g, wl, z0, r0, sweep, tag, slot, field4, up_rank, dn_rank); break;
          }
        }
        sync_slabs<S>();
        continue;
      }
#pragma unroll 1
      for (int item = tid; ok && item < items; item += nt) {
        const int wl = item % WC, grp = item / WC;
        const int zl = wl / P, iw = wl % P;
        const int z = z0 + zl;
        if (!RFIM_DCHECK(xa.err, grp * GT < gact && zl < PZ && iw < P, kDbgLattice)) continue;
        const int64_t wq = (int64_t)z * P + iw;
        float4 hh4[8] = {};
        if (!BIM) {
#pragma unroll
          for (int j = 0; j < 8; ++j) hh4[j] = __ldg(field4 + field4_index(c, wq, j, WPAD));
        }
        const uint32_t p0 = parity0_mask<L>(c, z, iw);
        uint32_t c0[GT], c1[GT], c2[GT], sf[GT], flip[GT];
#pragma unroll
        for (int gg = 0; gg < GT; ++gg) {
          const int g = min(grp * GT + gg, gact - 1);
          uint32_t nb[6];
          neighbour_words<L, S>(sp + ((size_t)g * 2 + (c ^ 1)) * WC, zl, iw, p0, up_rank, dn_rank, nb);
          count6(nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], c0[gg], c1[gg], c2[gg]);
          sf[gg] = sp[((size_t)g * 2 + c) * WC + wl];
          flip[gg] = 0u;
        }
        const uint32_t fb = BIM ? v.hbits[(int64_t)c * W + wq] : 0u;
        PairSlices ps[GT];
#pragma unroll
        for (int gg = 0; gg < GT; ++gg) ps[gg] = make_pairs(c0[gg], c1[gg], c2[gg], sf[gg], fb);
        // replicas past the end of a partial group repeat the last one; only their write is skipped.
        // Float field: flip = fk[k] << 8k once all blocks are done.
        uint32_t fk[GT][4];
#pragma unroll
        for (int gg = 0; gg < GT; ++gg)
#pragma unroll
          for (int k = 0; k < 4; ++k) fk[gg][k] = 0u;
#pragma unroll kBlockUnroll
        for (int jj = 0; jj < 8; ++jj) {
          const int j = 7 - jj;
#pragma unroll
          for (int gg = 0; gg < GT; ++gg) {
            const int g = min(grp * GT + gg, gact - 1);
            const Words4 w = philox10(v.seed, v.realization, (uint32_t)(8 * wq + j), (uint32_t)(r0 + g), sweep, tag);
            decide_block<BIM>(w, ps[gg], j, slot0 + (uint32_t)g * kTabSlot, hh4[j], flip[gg], fk[gg]);
          }
        }
        if (!BIM) {
#pragma unroll
          for (int gg = 0; gg < GT; ++gg) flip[gg] = fk[gg][0] | (fk[gg][1] << 8) | (fk[gg][2] << 16) | (fk[gg][3] << 24);
        }
#pragma unroll
        for (int gg = 0; gg < GT; ++gg) {
          const int g = grp * GT + gg;
          if (GT > 1 && g >= gact) continue;
          sp[((size_t)g * 2 + c) * WC + wl] = sf[gg] ^ flip[gg];
        }
      }
      sync_slabs<S>();
    }
  }

  for (int t = tid; ok && t < gact * 2 * WC; t += nt) {
    const int g = t / (2 * WC), rem = t % (2 * WC), c = rem / WC, wl = rem % WC;
    const int64_t gw = ((int64_t)(r0 + g) * 2 + c) * W + (int64_t)z0 * P + wl;
    if (I8)
      unpack_int8_word(sp[t], v.spins8 + 32 * gw);
    else
      v.bits[gw] = sp[t];
  }
  if (xa.enabled) interval_tail<L, S, BIM, XI>(v, G, r0, ok ? gact : 0, rank, nsw, field4, xa);
}

template <int L, int S, int GT, bool BIM, int NT, bool I8 = false, int NS = 1>
__global__ void __launch_bounds__(NT) k_sweeps_bits(RealView v, int32_t G, uint32_t sweep0, int32_t nsw,
                                                     const float4 *__restrict__ field4, ExchArgs xa) {
  const int rank = S > 1 ? (int)cluster_rank() : 0;
  const int r0 = (int)(blockIdx.x / S) * G;
  const int gact = min(G, v.R - r0);
  xa.expected = gridDim.x;
  bits_interval<L, S, GT, BIM, false, I8, NS>(v, G, r0, gact, rank, sweep0, nsw, field4, xa);
}

}  // namespace rfim
