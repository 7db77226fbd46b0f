// Grid-wide bit-layout sweep: one cooperative launch with one CTA per SM covers every SM, whatever
// the replica count.  Same arithmetic and decisions as kernels_bits.cuh.  A thread item is one
// 32-site word of GTI replicas of a group (GTI = 4: the field of the word is loaded once for the
// group; GTI = 1: four times more, smaller items, so that the items of a CTA split into nearly
// whole rounds of its threads).
//
// The realization's (4-replica group, z plane) units are split evenly over the CTAs
// (grid_partition.cuh); each CTA keeps its planes of both colours in shared memory for the whole
// exchange interval.  The z neighbours of a piece's end planes live in other CTAs.  Each
// half-sweep updates the end planes first (in the first rounds of thread items), writes them to
// the global lattice as they are done and releases the CTA's progress word; the interior planes
// follow.  During the last round, warps without an item acquire the neighbours' progress words
// and load their end planes (L2) for the next half-sweep, so the neighbours have normally
// published long before they are needed.  With the fused exchange a launch runs up to n_iv
// exchange intervals: after each interval's energy partials all CTAs meet at an arrival count,
// and every CTA takes the exchange step on its own copy of the temperature assignment.  Waits are
// bounded (expiry sets the kernel's error word and every later wait returns at once); the kernel
// always terminates.
#pragma once
#include <cstdint>

#include "grid_partition.cuh"
#include "kernels_bits.cuh"

namespace rfim {

constexpr unsigned kGridSpinLimit = 1u << 22;

struct GridArgs {
  GridPart gp;
  unsigned int *prog;  // [P] prog_base + half-sweeps completed by each CTA in this launch
  uint32_t prog_base;  // every word's value when the launch starts
  // exchange intervals in this launch (with the fused exchange); after each interval's partials
  // every CTA adds one to *arrive and waits for arrive_base + P (interval + 1) arrivals
  int32_t n_iv;
  uint32_t arrive_base;
  unsigned int *arrive;
  int32_t rcap;  // replica capacity: partials are [2 intervals][rcap][slots]
  int32_t max_units;   // units of the largest CTA (shared-memory sizing)
  int32_t slots;       // partial-sum slots per replica (CTAs sharing one group, at most)
  long long *partB, *partM, *partFi;  // [Rcap][slots]
  double *partF;
};

// Shared-memory exchange state every CTA of the grid-wide kernel keeps: t2r, r2t (int32), E
// (double), M (int64) for rcap replicas, 8-byte aligned.
__host__ __device__ constexpr size_t grid_xs_bytes(int rcap) { return (size_t)rcap * 24 + 16; }

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait for prog[k] >= need; false on expiry (which is recorded) or an earlier expiry.
__device__ __forceinline__ bool grid_wait(const unsigned *prog, int k, unsigned need, unsigned *err,
                                          unsigned limit = kGridSpinLimit) {
  for (unsigned it = 0; it < limit; ++it) {
    if (ld_acquire_u32(prog + k) >= need) return true;
    if (*(volatile unsigned *)err) return false;
    __nanosleep(64);
  }
  atomicOr(err, 2u);
  return false;
}

// Hot loop of a round range of a half-sweep of the grid-wide kernel, kept out of line so that
// its register allocation does not carry the kernel's set-up and schedule state.
struct GridHot {
  uint32_t *lat;
  const float4 *field4;
  uint32_t *bits;
  const uint32_t *hbits;
  uint32_t seed, realization, slot0;
  int nb_items, np;
  unsigned *err;
  const uint32_t *desc;
  const uint8_t *order;
  const Piece *pc;
  const int32_t *pcs, *pgact;
};

template <int L, bool BIM, int GG, int GTI>
__device__ __noinline__ void grid_process(const GridHot *hot_s, int i0, int i1, int c, uint32_t sweep, uint32_t tag) {
  const GridHot hot = *hot_s;  // from shared memory: the caller keeps none of it in registers
  constexpr int PW = L * L / 64, W = L * L * L / 64;
  constexpr int64_t WPAD = (W + 31) / 32 * 32;
  constexpr int IPW = PW * (GG / GTI);
  const int nt = blockDim.x, tid = threadIdx.x, other = c ^ 1;
  const float4 *__restrict__ field4 = hot.field4;
#pragma unroll 1
  for (int it = i0 + tid; it < i1; it += nt) {
    const uint32_t d = hot.desc[hot.order[it / IPW]];
    const int w = it % PW;
    const bool end_plane = it < hot.nb_items;
    const int gb = (it % IPW) / PW * GTI;  // first replica of this item within the group
    const int p = (int)(d >> 26), zl = (int)((d >> 18) & 255u);
    if (!RFIM_DCHECK(hot.err, p < hot.np && zl < hot.pc[p].n, kDbgPartition)) continue;
    const int z = hot.pc[p].z0 + zl;
    const int64_t wq = (int64_t)z * PW + w;
    const int gact = hot.pgact[p], cs = hot.pcs[p];
    if (gb >= gact) continue;  // GTI = 1: replica past the end of a partial group
    uint32_t *Pl = hot.lat + (d & 0x3FFFFu) + (zl + 1) * PW;  // plane zl of replica 0, colour 0
    float4 hh4[8] = {};
    if (!BIM) {
#pragma unroll
      for (int j = 0; j < 8; ++j) hh4[j] = __ldg(field4 + field4_index(c, wq, j, WPAD));
    }
    const uint32_t p0 = parity0_mask<L>(c, z, w);
    PairSlices ps[GTI];
    uint32_t sf[GTI], flip[GTI], fk[GTI][4];
    const uint32_t fb = BIM ? hot.hbits[(int64_t)c * W + wq] : 0u;
#pragma unroll
    for (int gg = 0; gg < GTI; ++gg) {
      const int g = min(gb + gg, gact - 1);
      const uint32_t *O = Pl + (g * 2 + other) * cs;
      uint32_t nbw[6], c0, c1, c2;
      nb_xy<L>(O[w], O[(w + 1) % PW], O[(w + PW - 1) % PW], p0, nbw[0], nbw[1], nbw[2], nbw[3]);
      nbw[4] = O[PW + w];
      nbw[5] = O[w - PW];
      count6(nbw[0], nbw[1], nbw[2], nbw[3], nbw[4], nbw[5], c0, c1, c2);
      sf[gg] = Pl[(g * 2 + c) * cs + w];
      ps[gg] = make_pairs(c0, c1, c2, sf[gg], fb);
      flip[gg] = 0u;
#pragma unroll
      for (int q = 0; q < 4; ++q) fk[gg][q] = 0u;
    }
    const int r0 = hot.pc[p].g * GG;
#pragma unroll kBlockUnroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = 7 - jj;
#pragma unroll
      for (int gg = 0; gg < GTI; ++gg) {
        const int g = min(gb + gg, gact - 1);
        const Words4 wd = philox10(hot.seed, hot.realization, (uint32_t)(8 * wq + j), (uint32_t)(r0 + g), sweep, tag);
        decide_block<BIM>(wd, ps[gg], j, hot.slot0 + (uint32_t)(p * GG + g) * kTabSlot, hh4[j], flip[gg], fk[gg]);
      }
    }
#pragma unroll
    for (int gg = 0; gg < GTI; ++gg) {
      if (gb + gg >= gact) continue;
      if (!BIM) flip[gg] = fk[gg][0] | (fk[gg][1] << 8) | (fk[gg][2] << 16) | (fk[gg][3] << 24);
      const uint32_t nw = sf[gg] ^ flip[gg];
      Pl[((gb + gg) * 2 + c) * cs + w] = nw;
      if (end_plane) hot.bits[((int64_t)(r0 + gb + gg) * 2 + c) * W + wq] = nw;  // publish
    }
  }
}

// I8: the realization lives in the int8 layout (v.spins8); the CTA packs its pieces and the first
// halos from bytes and unpacks its pieces at the end, and v.bits is a scratch array in the bit
// layout that carries only the end planes published during the launch.
template <int L, bool BIM, int GG, int GTI, int NT, bool I8 = false>
__global__ void __launch_bounds__(NT, 1) k_sweeps_grid(RealView v, GridArgs ga, uint32_t sweep0, int32_t nsw,
                                                        const float4 *__restrict__ field4, ExchArgs xa) {
  constexpr int PW = L * L / 64, W = L * L * L / 64;
  constexpr int64_t WPAD = (W + 31) / 32 * 32;
  extern __shared__ __align__(16) uint32_t sm[];
  const int k = blockIdx.x, nt = blockDim.x, tid = threadIdx.x;
  // Shared-memory lattice: per piece p a region [GG replicas][2 colours][n_p + 2 planes][PW words]
  // whose planes 0 and n_p + 1 are the z halos (the neighbouring CTAs' end planes), so that the
  // z neighbours of every local plane are the planes before and after it.
  __shared__ Piece pc[kGridMaxPieces];
  __shared__ int32_t pbase[kGridMaxPieces], pcs[kGridMaxPieces], pgact[kGridMaxPieces];
  __shared__ int np_s, nu_s, nb_s;
  __shared__ uint32_t udesc[256];  // per local unit: region base (words) | plane in piece << 18 | piece << 26
  __shared__ uint8_t order[256];   // local units: piece end planes first, then interior
  if (tid == 0) {
    Piece tmp[kGridMaxPieces];
    const int np = grid_pieces(ga.gp, k, tmp);
    int nu = 0, base = 0;
    for (int p = 0; p < np; ++p) {
      pc[p] = tmp[p];
      pbase[p] = base;
      pcs[p] = (tmp[p].n + 2) * PW;
      pgact[p] = min(GG, v.R - tmp[p].g * GG);
      for (int i = 0; i < tmp[p].n && tmp[p].lu0 + i < 256; ++i)
        udesc[tmp[p].lu0 + i] = (uint32_t)base | ((uint32_t)i << 18) | ((uint32_t)p << 26);
      base += GG * 2 * (tmp[p].n + 2) * PW;
      nu += tmp[p].n;
    }
    int o = 0;
    for (int p = 0; p < np; ++p) {
      order[o++] = (uint8_t)tmp[p].lu0;
      if (tmp[p].n > 1) order[o++] = (uint8_t)(tmp[p].lu0 + tmp[p].n - 1);
    }
    const int nend = o;
    for (int p = 0; p < np; ++p)
      for (int i = 1; i + 1 < tmp[p].n; ++i) order[o++] = (uint8_t)(tmp[p].lu0 + i);
    np_s = np;
    nu_s = nu;
    nb_s = nend;
  }
  __syncthreads();
  // debug build: the partition must fit the shared-memory plan (pieces, planes, local order)
  const bool part_ok = RFIM_DCHECK(xa.err, np_s >= 1 && np_s <= kGridMaxPieces && nu_s <= ga.max_units && nu_s <= 255 &&
                                               nb_s <= nu_s,
                                   kDbgPartition);
  const int np = part_ok ? np_s : 0, nu = part_ok ? nu_s : 0, nb = part_ok ? nb_s : 0;
  uint32_t *lat = sm;                                                   // piece regions
  uint32_t *tab = lat + (size_t)(ga.max_units + 2 * kGridMaxPieces) * GG * 2 * PW;  // [pieces][GG] table slots
  const uint32_t slot0 = tab_slot0(tab);
  // exchange state, after the table slots (tab_bytes includes the slots' alignment slack)
  char *xs = reinterpret_cast<char *>(tab) + tab_bytes(kGridMaxPieces * GG);
  xs += (8u - ((uintptr_t)xs & 7u)) & 7u;
  double *E_s = reinterpret_cast<double *>(xs);
  long long *M_s = reinterpret_cast<long long *>(E_s + ga.rcap);
  int32_t *t2r_s = reinterpret_cast<int32_t *>(M_s + ga.rcap);
  int32_t *r2t_s = t2r_s + ga.rcap;
  if (xa.enabled)
    for (int r = tid; r < v.R; r += nt) {
      t2r_s[r] = v.t2r[r];
      r2t_s[r] = v.r2t[r];
    }
  // word w of plane zl (-1 .. n_p: halos included) of colour c of replica gg in piece p
  auto at = [&](int p, int gg, int c, int zl) { return lat + pbase[p] + (gg * 2 + c) * pcs[p] + (zl + 1) * PW; };

  for (int t = tid; t < nu * GG * 2 * PW; t += nt) {
    const int lu = t / (GG * 2 * PW), rem = t % (GG * 2 * PW), gg = rem / (2 * PW), c = (rem / PW) & 1, w = rem % PW;
    const uint32_t d = udesc[lu];
    const int p = (int)(d >> 26), zl = (int)((d >> 18) & 255u);
    const int r = pc[p].g * GG + gg, z = pc[p].z0 + zl;
    const int64_t gw = ((int64_t)r * 2 + c) * W + (int64_t)z * PW + w;
    at(p, gg, c, zl)[w] = r < v.R ? (I8 ? pack_int8_word(v.spins8 + 32 * gw) : v.bits[gw]) : 0u;
  }
  tab_fill<BIM>(v, tab, slot0, np * GG, [&](int t) { return min(pc[t / GG].g * GG + t % GG, v.R - 1); });
  __syncthreads();

  constexpr int IPW = PW * (GG / GTI);  // items per plane
  const int items = nu * IPW;
  // rounds of nt items that hold every end-plane item, and the first item of the last round
  const int split = min(items, (nb * IPW + nt - 1) / nt * nt);
  const int last_round = items > split ? split + (items - split - 1) / nt * nt : items;
  const int warp = tid >> 5, busy_warps = (items - last_round + 31) / 32;
  const int idle_warps = items > split ? nt / 32 - busy_warps : 0;
  unsigned *err = xa.err;

  // Loads the colour-`other` end planes of every piece's z neighbours into its halo planes once
  // their CTAs have published `need` half-sweeps: thread `lead` waits, the group of `count`
  // threads (whole warps, named barrier `bar`) holding it then loads.  The caller makes the loads
  // visible with a CTA barrier.
  // from_bytes: the int8 layout as the launch found it (the first halos of an I8 launch)
  auto fetch_halos = [&](int other, unsigned need, int t0, int count, int bar, bool from_bytes = false) {
    const int lt = tid - t0;
    if (lt == 0) {
      for (int p = 0; p < np; ++p) {
        const int64_t base = (int64_t)pc[p].g * L;
        int klo = grid_owner(ga.gp, base + (pc[p].z0 + L - 1) % L);
        int khi = grid_owner(ga.gp, base + (pc[p].z0 + pc[p].n) % L);
        if (!RFIM_DCHECK(err, klo >= 0 && klo < ga.gp.P && khi >= 0 && khi < ga.gp.P, kDbgPartition)) klo = khi = k;
        grid_wait(ga.prog, klo, need, err);
        grid_wait(ga.prog, khi, need, err);
      }
    }
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(count) : "memory");
    for (int t = lt; t < np * 2 * GG * PW; t += count) {
      const int p = t / (2 * GG * PW), side = (t / (GG * PW)) & 1, gg = (t / PW) % GG, w = t % PW;
      const int r = min(pc[p].g * GG + gg, v.R - 1);
      const int z = side ? (pc[p].z0 + pc[p].n) % L : (pc[p].z0 + L - 1) % L;
      const int64_t gw = ((int64_t)r * 2 + other) * W + (int64_t)z * PW + w;
      at(p, gg, other, side ? pc[p].n : -1)[w] = from_bytes ? pack_int8_word(v.spins8 + 32 * gw) : __ldcg(v.bits + gw);
    }
  };
  // the neighbours' colour-1 end planes as the launch found them
  fetch_halos(1, ga.prog_base, 0, nt, 1, I8);
  __shared__ GridHot hot;
  if (tid == 0) {
    hot.lat = lat;
    hot.field4 = field4;
    hot.bits = v.bits;
    hot.hbits = v.hbits;
    hot.seed = v.seed;
    hot.realization = v.realization;
    hot.slot0 = slot0;
    hot.nb_items = nb * IPW;
    hot.np = np;
    hot.err = err;
    hot.desc = udesc;
    hot.order = order;
    hot.pc = pc;
    hot.pcs = pcs;
    hot.pgact = pgact;
  }
  __syncthreads();

  // Several exchange intervals per launch (fused exchange, ga.n_iv > 1): every CTA takes each
  // interval's exchange step itself (below) and refills its decision tables from its own copy of
  // the new temperature assignment.
  const int n_iv = xa.enabled ? max(ga.n_iv, 1) : 1;
  for (int iv = 0; iv < n_iv; ++iv) {
    const unsigned pbase = ga.prog_base + (unsigned)(2 * nsw * iv);
    if (iv > 0) {
      // tables of the temperatures the previous exchange step assigned
      tab_fill_temps<BIM>(v, tab, slot0, np * GG, [&](int t) { return r2t_s[min(pc[t / GG].g * GG + t % GG, v.R - 1)]; });
      __syncthreads();
    }
    for (int h = 0; h < 2 * nsw; ++h) {
      const int c = h & 1, other = c ^ 1;
      const uint32_t sweep = sweep0 + (uint32_t)(iv * nsw + (h >> 1));
      const uint32_t tag = tag_word(kTagMetro, v.stage, (uint32_t)c);
      auto process = [&](int i0, int i1) {
        grid_process<L, BIM, GG, GTI>(&hot, i0, i1, c, sweep, tag);
      };
      // end planes (and the interior items sharing their rounds), then the progress word: the CTA
      // barrier orders every thread's end-plane stores before thread 0's gpu-scope fence and release
      // (cumulativity), as in a grid-wide barrier
      process(0, split);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release_u32(ga.prog + k, pbase + (unsigned)(h + 1));
      }
      // interior planes; warps without an item in the last round fetch the halos of the next
      // half-sweep (this colour's end planes of the neighbours), else every thread does afterwards
      process(split, items);
      if (idle_warps > 0) {
        if (warp >= nt / 32 - idle_warps) fetch_halos(c, pbase + (unsigned)(h + 1), nt - 32 * idle_warps, 32 * idle_warps, 1);
      } else {
        __syncthreads();
        fetch_halos(c, pbase + (unsigned)(h + 1), 0, nt, 1);
      }
      __syncthreads();
    }

    if (iv == n_iv - 1) {  // the lattice back to global memory once, after the last interval
      for (int t = tid; t < nu * GG * 2 * PW; t += nt) {
        const int lu = t / (GG * 2 * PW), rem = t % (GG * 2 * PW), gg = rem / (2 * PW), c = (rem / PW) & 1, w = rem % PW;
        const uint32_t d = udesc[lu];
        const int p = (int)(d >> 26), zl = (int)((d >> 18) & 255u);
        const int r = pc[p].g * GG + gg, z = pc[p].z0 + zl;
        const int64_t gw = ((int64_t)r * 2 + c) * W + (int64_t)z * PW + w;
        if (r < v.R) {
          if (I8)
            unpack_int8_word(at(p, gg, c, zl)[w], v.spins8 + 32 * gw);
          else
            v.bits[gw] = at(p, gg, c, zl)[w];
        }
      }
    }
    if (!xa.enabled) return;

    // ---- energy partials (Eq. 1) per (replica, piece), then the exchange tail ----------------
    // (the colour-1 halo planes hold the neighbours' final end planes, fetched by the last half-sweep).
    // As in the cluster plan's tail: up to RB replicas of a piece at a time (one field load per word
    // for all of them, one barrier pair, then one warp per replica over the warps' partials); the
    // float field term as exact fixed-point sums from the field limbs when given, else error-free
    // float sums.
    constexpr int RB = GG < kTailRB ? GG : kTailRB;
    __shared__ int red_i[BIM ? 3 : 2][RB][32];
    __shared__ long long red_l[BIM ? 1 : RB][32];
    __shared__ double red_d[RB][32];
    const int lane = tid & 31, wid = tid >> 5, nw = (nt + 31) >> 5;
    const bool limbs = !BIM && xa.flimb != nullptr;
    for (int p = 0; p < np; ++p) {
      const int gact = pgact[p], nwd = pc[p].n * PW;
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
        for (int t = tid; t < 2 * nwd; t += nt) {
          const int c = t / nwd, rem = t % nwd, pl = rem / PW, w = rem % PW;
          const int z = pc[p].z0 + pl;
          const int64_t wq = (int64_t)z * PW + w;
          const uint32_t hb = BIM ? v.hbits[(int64_t)c * W + wq] : 0u;
          uint32_t self[RB];
  #pragma unroll
          for (int gg = 0; gg < RB; ++gg) {
            self[gg] = gg < ng ? at(p, g0 + gg, c, pl)[w] : 0u;
            if (gg >= ng) continue;
            m[gg] += 2 * __popc(self[gg]) - 32;
            if (c == 0) {
              const uint32_t *O = at(p, g0 + gg, 1, pl);
              uint32_t nbw[6];
              nb_xy<L>(O[w], O[(w + 1) % PW], O[(w + PW - 1) % PW], parity0_mask<L>(0, z, w), nbw[0], nbw[1], nbw[2],
                       nbw[3]);
              nbw[4] = O[PW + w];
              nbw[5] = O[w - PW];
  #pragma unroll
              for (int d = 0; d < 6; ++d) b[gg] += 32 - 2 * __popc(self[gg] ^ nbw[d]);
            }
            if (BIM) fi[gg] += 32 - 2 * __popc(self[gg] ^ hb);
          }
          if (limbs) {
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
                hs[gg] = __dp4a((int)up, (int)top[j], hs[gg]);
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
                for (int q = 0; q < 4; ++q) {
                  const float term = ((self[gg] >> (8 * q + j)) & 1u) ? hk[q] : -hk[q];
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
          if constexpr (BIM) {
            const int tf = warp_reduce_sum(fi[gg]);
            if (lane == 0) red_i[BIM ? 2 : 0][gg][wid] = tf;
          } else {
            long long fl = 0;
            if (limbs)
              fl = (long long)hu[gg][0] + ((long long)hu[gg][1] << 8) + ((long long)hu[gg][2] << 16) +
                   ((long long)hu[gg][3] << 24) + ((long long)hs[gg] << 32);
            const long long tf = warp_reduce_sum(fl);
            if (lane == 0) red_l[BIM ? 0 : gg][wid] = tf;
          }
          const double td = (BIM || limbs) ? 0.0 : warp_reduce_sum((double)fs[gg] + (double)fe[gg]);
          if (lane == 0) {
            red_i[0][gg][wid] = tb;
            red_i[1][gg][wid] = tm;
            red_d[gg][wid] = td;
          }
        }
        __syncthreads();
        if (wid < ng) {  // warp gg adds the warps' partials of replica g0 + gg of the piece
          const int gg = wid;
          const long long tb = warp_reduce_sum(lane < nw ? (long long)red_i[0][gg][lane] : 0LL);
          const long long tm = warp_reduce_sum(lane < nw ? (long long)red_i[1][gg][lane] : 0LL);
          const long long tf =
              warp_reduce_sum(lane < nw ? (BIM ? (long long)red_i[BIM ? 2 : 0][gg][lane] : red_l[BIM ? 0 : gg][lane]) : 0LL);
          const double td = warp_reduce_sum(lane < nw ? red_d[gg][lane] : 0.0);
          if (lane == 0) {
            const int slab = grid_slab_of(ga.gp, k, pc[p].g);
            const int r = pc[p].g * GG + g0 + gg;
            const int64_t slot = ((int64_t)(iv & 1) * ga.rcap + r) * ga.slots + slab;
            if (RFIM_DCHECK(xa.err, slab >= 0 && slab < ga.slots && r < v.R, kDbgPartition)) {
              ga.partB[slot] = tb;
              ga.partM[slot] = tm;
              ga.partFi[slot] = tf;
              ga.partF[slot] = td;
            }
          }
        }
        __syncthreads();
      }
    }
    // Every CTA takes exchange step j + iv itself: after all P CTAs have arrived with their
    // partials, each sums every replica's energy (Eq. 1) in the same order and takes the same
    // decisions on its own copy of the temperature assignment; CTA 0 alone keeps the global state
    // (counts, measurement, and the assignment and energies after the launch's last step).  The
    // partials alternate between two buffers, so a CTA already in the next interval does not
    // overwrite sums that a slower one is still reading.
    if (tid == 0) {
      __threadfence();
      atomicAdd(ga.arrive, 1u);
      grid_wait(ga.arrive, 0, ga.arrive_base + (unsigned)gridDim.x * (unsigned)(iv + 1), err);
    }
    __syncthreads();
    const uint32_t jx = xa.j + (uint32_t)iv;
    const int64_t pb = (int64_t)(iv & 1) * ga.rcap;
    for (int r = tid; r < v.R; r += nt) {
      const int g = r / GG;
      const int nslab = grid_owner(ga.gp, (int64_t)g * L + L - 1) - grid_owner(ga.gp, (int64_t)g * L) + 1;
      long long tb = 0, tm = 0, tf = 0;
      double td = 0.0;
      for (int q = 0; q < nslab; ++q) {
        const int64_t slot = (pb + r) * ga.slots + q;
        tb += __ldcg(ga.partB + slot);
        tm += __ldcg(ga.partM + slot);
        tf += __ldcg(ga.partFi + slot);
        td += __ldcg(ga.partF + slot);
      }
      const double F = BIM ? xa.h * (double)tf
                           : (xa.flimb ? ldexp((double)(2 * tf - xa.fquant->Htot), xa.fquant->qe) : td);
      E_s[r] = -xa.J * (double)tb - F;
      M_s[r] = tm;
    }
    __syncthreads();
    for (int pr = tid;; pr += nt) {
      const int32_t kk = (int32_t)(jx & 1u) + 2 * pr;
      if (kk + 1 >= v.R) break;
      const int32_t a = t2r_s[kk], b = t2r_s[kk + 1];
      const bool accept = exchange_accept(v, jx, kk, E_s[a], E_s[b]);
      if (k == 0) {
        v.att[kk] += 1;
        if (accept) v.acc[kk] += 1;
      }
      if (accept) {
        t2r_s[kk] = b;
        t2r_s[kk + 1] = a;
        r2t_s[b] = kk;
        r2t_s[a] = kk + 1;
      }
    }
    __syncthreads();
    if (k == 0) {
      if ((int64_t)jx >= xa.measure_from) {
        const double Nd = (double)v.N;
        for (int kk = tid; kk < v.R; kk += nt) {
          const int32_t a = t2r_s[kk];
          measure_add(v.obs + (int64_t)kk * 5, E_s[a], M_s[a], Nd);
        }
        if (tid == 0) *v.n_meas += 1;
      }
      if (iv == n_iv - 1)
        for (int r = tid; r < v.R; r += nt) {
          v.t2r[r] = t2r_s[r];
          v.r2t[r] = r2t_s[r];
          v.E[r] = E_s[r];
          v.M[r] = M_s[r];
        }
    }
    __syncthreads();
  }  // exchange intervals
}

}  // namespace rfim
