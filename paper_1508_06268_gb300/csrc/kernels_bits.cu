// Launch plan, dispatch and helpers of the bit-layout sweep kernel (kernels_bits.cuh).
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kernels_bits.cuh"
#include "kernels_grid.cuh"
#include "kernels_mh.cuh"
#include "lattice.cuh"
#include "sweep_bits.h"

namespace rfim {

cudaError_t raise_smem_limit(const void *fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> limit;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t &cur = limit[{dev, fn}];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

namespace {

using KernelFn = void (*)(RealView, int32_t, uint32_t, int32_t, const float4 *, ExchArgs);

template <int L, int S, int GT, int NT>
KernelFn pick(bool bim) {
  return bim ? (KernelFn)k_sweeps_bits<L, S, GT, true, NT> : (KernelFn)k_sweeps_bits<L, S, GT, false, NT>;
}

// Instances available to launch plans (L, cluster size S, replicas per thread GT, threads NT);
// i8: the int8-layout staging instances (kernels_bits_i8.cu), default shapes only.
KernelFn kernel_for(int L, int S, int GT, int NT, bool bim, bool i8 = false, int ns = 1) {
  if (i8) return ns == 1 ? (KernelFn)kernel_for_i8(L, S, GT, NT, bim) : nullptr;
  if (ns == 4) return (KernelFn)kernel_for_split(L, S, GT, NT, bim);
  if (ns != 1) return nullptr;
#define RFIM_BITS_INSTANCE(l, s_, gt, nt) \
  if (L == l && S == s_ && GT == gt && NT == nt) return pick<l, s_, gt, nt>(bim);
  RFIM_BITS_INSTANCE(64, 1, 1, 512)
  RFIM_BITS_INSTANCE(64, 1, 1, 1024)
  RFIM_BITS_INSTANCE(64, 1, 2, 512)
  RFIM_BITS_INSTANCE(64, 2, 1, 1024)
  RFIM_BITS_INSTANCE(64, 2, 2, 512)
  RFIM_BITS_INSTANCE(64, 2, 2, 1024)
  RFIM_BITS_INSTANCE(64, 4, 1, 1024)
  RFIM_BITS_INSTANCE(64, 4, 2, 512)
  RFIM_BITS_INSTANCE(64, 4, 2, 1024)
  RFIM_BITS_INSTANCE(64, 4, 4, 512)
  RFIM_BITS_INSTANCE(64, 4, 4, 1024)
  RFIM_BITS_INSTANCE(32, 1, 1, 512)
  RFIM_BITS_INSTANCE(32, 1, 2, 512)
  RFIM_BITS_INSTANCE(32, 2, 1, 512)
  RFIM_BITS_INSTANCE(32, 2, 1, 256)
  RFIM_BITS_INSTANCE(32, 4, 1, 128)
  RFIM_BITS_INSTANCE(16, 1, 1, 512)
  RFIM_BITS_INSTANCE(8, 1, 1, 128)
  RFIM_BITS_INSTANCE(8, 1, 1, 512)
#undef RFIM_BITS_INSTANCE
  return nullptr;
}

using MhFn = void (*)(RealView, int32_t, uint32_t, int32_t, const float4 *, ExchArgs, MultiHit);

template <int L, int S, int GT, int NT, int T>
MhFn mh_pick(bool bim) {
  return bim ? (MhFn)k_sweeps_bits_mh<L, S, GT, true, NT, T> : (MhFn)k_sweeps_bits_mh<L, S, GT, false, NT, T>;
}

// Multi-hit instances: the default cluster / single-CTA shapes of L = 64, 32, 16, per tile edge.
MhFn mh_kernel_for(int L, int S, int GT, int NT, bool bim, int T) {
  if (L == 64 && S == 4 && GT == 4 && NT == 512)
    return T == 8 ? mh_pick<64, 4, 4, 512, 8>(bim) : T == 16 ? mh_pick<64, 4, 4, 512, 16>(bim)
                                                   : T == 32 ? mh_pick<64, 4, 4, 512, 32>(bim) : nullptr;
  if (L == 32 && S == 2 && GT == 1 && NT == 256)
    return T == 8 ? mh_pick<32, 2, 1, 256, 8>(bim) : T == 16 ? mh_pick<32, 2, 1, 256, 16>(bim) : nullptr;
  if (L == 16 && S == 1 && GT == 1 && NT == 512) return T == 8 ? mh_pick<16, 1, 1, 512, 8>(bim) : nullptr;
  return nullptr;
}

int words_per_cta(int L, int S) { return L <= 0 || S <= 0 ? 0 : (L / S) * (L * L / 64); }

using GridFn = void (*)(RealView, GridArgs, uint32_t, int32_t, const float4 *, ExchArgs);

template <int L, int GG, int GTI, int NT, bool I8 = false>
GridFn grid_pick(bool bim) {
  return bim ? (GridFn)k_sweeps_grid<L, true, GG, GTI, NT, I8> : (GridFn)k_sweeps_grid<L, false, GG, GTI, NT, I8>;
}

// Grid-wide instances: G replicas per unit, GT of them per thread item (GT = G: one field load
// per group); NT is the launch-bounds thread count (plans may launch fewer threads, in multiples
// of 32).
GridFn grid_kernel_for(int L, int G, int GT, int threads, bool bim, bool i8) {
  if (i8)  // the int8 layout staged as bits: the default shape only
    return L == 64 && G == 4 && GT == 4 && threads > 256 && threads <= 512 ? grid_pick<64, 4, 4, 512, true>(bim) : nullptr;
  if (threads <= 512) {
    if (L == 64 && G == 4 && GT == 4) return grid_pick<64, 4, 4, 512>(bim);
    if (L == 64 && G == 4 && GT == 1) return grid_pick<64, 4, 1, 512>(bim);
    if (L == 64 && G == 8 && GT == 8) return grid_pick<64, 8, 8, 512>(bim);
    if (L == 64 && G == 8 && GT == 4) return grid_pick<64, 8, 4, 512>(bim);
    if (L == 32 && G == 4 && GT == 4) return grid_pick<32, 4, 4, 512>(bim);
    if (L == 32 && G == 4 && GT == 1) return grid_pick<32, 4, 1, 512>(bim);
  } else if (threads <= 896) {
    if (L == 64 && G == 4 && GT == 2) return grid_pick<64, 4, 2, 896>(bim);
    if (L == 64 && G == 4 && GT == 4) return grid_pick<64, 4, 4, 896>(bim);
  }
  return nullptr;
}

constexpr size_t kGridMinSmem = 116 * 1024;  // more than half an SM's shared memory: one CTA per SM

// Partition of the current R over the CTAs of a grid-wide launch.
GridArgs grid_args(const BitsPlan &p, int32_t R, int sms) {
  GridArgs ga{};
  ga.gp.L = p.L;
  ga.gp.NG = (R + p.G - 1) / p.G;
  ga.gp.U = (int64_t)ga.gp.NG * p.L;
  int64_t P = std::min<int64_t>(sms, ga.gp.U / 3);
  if (P < 1) P = 1;
  ga.gp.P = (int32_t)P;
  int maxu = 0, slots = 0;
  for (int k = 0; k < ga.gp.P; ++k) maxu = std::max<int>(maxu, (int)(grid_begin(ga.gp, k + 1) - grid_begin(ga.gp, k)));
  for (int g = 0; g < ga.gp.NG; ++g)
    slots = std::max(slots, grid_owner(ga.gp, (int64_t)g * p.L + p.L - 1) - grid_owner(ga.gp, (int64_t)g * p.L) + 1);
  ga.max_units = maxu;
  ga.slots = slots;
  ga.prog = p.prog;
  ga.prog_base = 0;
  ga.n_iv = 1;
  ga.arrive_base = 0;
  ga.arrive = p.counter ? p.counter + 2 : nullptr;
  ga.rcap = p.Rcap;
  ga.partB = p.gpartB;
  ga.partM = p.gpartM;
  ga.partFi = p.gpartFi;
  ga.partF = p.gpartF;
  return ga;
}

size_t grid_smem(int L, int G, int max_units, int rcap) {
  const size_t PW = (size_t)L * L / 64;
  // piece regions with two halo planes each (both colours), the decision-table slots, then the
  // exchange state every CTA keeps (grid_xs_bytes)
  const size_t need = (size_t)(max_units + 2 * kGridMaxPieces) * G * 2 * PW * 4 + tab_bytes(kGridMaxPieces * G) +
                      grid_xs_bytes(rcap);
  return std::max(need, kGridMinSmem);
}

__global__ void k_build_field4(RealView v, float4 *field4, int64_t wpad) {
  const int64_t half = (int64_t)v.N / 2, W = half / 32;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * W * 8; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / (W * 8));
    const int64_t wq = (t / 8) % W;
    const int j = (int)(t % 8);
    const float *h = v.hh_c + c * half + wq * 32 + 4 * j;
    field4[field4_index(c, wq, j, wpad)] = make_float4(h[0], h[1], h[2], h[3]);
  }
}

// Largest |hh_i| as float bits (non-negative floats order like their bits) into *fmax.
__global__ void k_field_absmax(RealView v, unsigned *fmax) {
  unsigned m = 0u;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < v.N; t += (int64_t)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(v.hh_c[t]) & 0x7FFFFFFFu);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(fmax, m);
}

// Fixed-point field of the energy tail: qe = E - 38 with E = floor(log2 max |hh|) (-127 when the
// maximum is zero or subnormal), so |hh| / 2^qe < 2^39.  H = rint(hh / 2^qe) is exact wherever hh
// is at least 2^(qe + 23) and rounded by at most 2^(qe - 1) below; one thread per four sites
// (colour, word, block j) writes their five byte limbs, and the lattice sum of H goes to Htot.
__global__ void k_field_limbs(RealView v, uint4 *flimb, FieldQuant *fz, int64_t wpad) {
  const unsigned mb = fz->fmax;
  const int E = mb < 0x00800000u ? -127 : (int)(mb >> 23) - 127;
  const int qe = E - 38;
  const int64_t half = (int64_t)v.N / 2, W = half / 32;
  long long hsum = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * W * 8; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / (W * 8));
    const int64_t wq = (t / 8) % W;
    const int j = (int)(t % 8);
    const float *h = v.hh_c + c * half + wq * 32 + 4 * j;
    uint32_t lo[4] = {0u, 0u, 0u, 0u}, top = 0u;
    for (int k = 0; k < 4; ++k) {
      const long long H = llrint(ldexp((double)h[k], -qe));
      hsum += H;
      const unsigned long long u = (unsigned long long)H;
      for (int l = 0; l < 4; ++l) lo[l] |= (uint32_t)((u >> (8 * l)) & 0xFFu) << (8 * k);
      top |= (uint32_t)((u >> 32) & 0xFFu) << (8 * k);  // two's complement: floor(H / 2^32) as a byte
    }
    flimb[flimb_index(c, wq, j, wpad)] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    reinterpret_cast<uint32_t *>(flimb + flimb_index(c, wq, 8 + j / 4, wpad))[j % 4] = top;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(0xffffffffu, hsum, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&fz->Htot), (unsigned long long)hsum);
  if (blockIdx.x == 0 && threadIdx.x == 0) fz->qe = qe;
}

}  // namespace

bool bits_supported(int32_t L) { return L == 8 || L == 16 || L == 32 || L == 64; }

bool multihit_tile_ok(int32_t L, int32_t tile) {
  return (L == 16 || L == 32 || L == 64) && (tile == 8 || tile == 16 || tile == 32) && L % (2 * tile) == 0;
}

MultiHit make_multihit(int32_t L, int32_t mh, int32_t tile) {
  MultiHit m;
  if (mh <= 0 || !multihit_tile_ok(L, tile)) return m;
  m.mh = mh;
  m.tile = tile;
  return m;
}

cudaError_t prepare_multihit(const BitsPlan &plan, bool bimodal) {
  if (plan.S == 0) return cudaErrorInvalidConfiguration;
  for (int T : {8, 16, 32}) {
    if (!multihit_tile_ok(plan.L, T)) continue;
    MhFn fn = mh_kernel_for(plan.L, plan.S, plan.GT, plan.threads, bimodal, T);
    if (!fn) return cudaErrorInvalidConfiguration;
    cudaError_t e = raise_smem_limit((const void *)fn, plan.smem);
    if (e == cudaSuccess && plan.S > 1)
      e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {
thread_local const char *t_plan_override = nullptr;
std::mutex g_tuned_mu;
std::map<std::tuple<int, int, bool>, std::string> g_tuned;  // (L, R, bimodal) -> "S,G,GT,threads"
}  // namespace

void set_plan_override(const char *plan) { t_plan_override = plan; }

void remember_tuned_plan(int32_t L, int32_t R, bool bimodal, const std::string &plan) {
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  g_tuned[{L, R, bimodal}] = plan;
}

std::vector<std::string> plan_candidates(int32_t L) {
  if (L == 64)
    return {"4,4,4,512", "0,4,4,512", "0,4,1,512", "4,4,2,512", "2,2,2,512", "4,4,4,1024", "1,1,1,1024"};
  if (L == 32)
    return {"2,1,1,256", "4,1,1,128", "1,1,1,512", "1,2,2,512", "2,1,1,512", "0,4,4,512", "0,4,1,512",
            "2,1,1,1024,4", "2,1,1,512,4", "4,1,1,512,4"};
  if (L == 16) return {"1,8,1,512", "1,4,1,512", "1,16,1,512", "1,8,1,1024,4", "1,4,1,512,4", "1,8,1,512,4"};
  return {"1,16,1,128", "1,16,1,512", "1,8,1,128", "1,16,1,512,4", "1,8,1,256,4"};
}

int make_bits_plan(int32_t L, int32_t Rcap, bool bimodal, BitsPlan *plan, std::string *err, bool i8) {
  BitsPlan p;
  p.L = L;
  p.Rcap = Rcap;
  p.i8 = i8;
  int sms_dev = 0;
  cudaDeviceGetAttribute(&sms_dev, cudaDevAttrMultiProcessorCount, 0);
  if (L == 64) {  // both layouts (the int8 one staged as bits)
    // clusters of 4 z slabs x 4 replicas, unless they would leave more than a fifth of the SMs
    // idle (e.g. R = 70 after adaptation: 72 CTAs) or need more clusters than fit at once (a
    // second wave; 36 clusters of 4 at one CTA per SM on GB300); then the grid-wide plan
    const int cluster_ctas = 4 * ((Rcap + 3) / 4);
    p.S = 4; p.G = 4; p.GT = 4; p.threads = 512;
    // grid-wide plan when clusters of 4 would leave an eighth of the SMs or more idle (measured at
    // L = 64, Gaussian field: R = 112 / 120 / 128 grid 945 / 954 / 999 against clusters 860 / 923 /
    // 984 attempts/ns; R = 136 / 144 clusters 1043 / 1104 against 987 / 922)
    bool grid = sms_dev > 0 && 8 * cluster_ctas <= 7 * sms_dev;
    if (!grid) {
      KernelFn cf = kernel_for(L, 4, 4, 512, bimodal);
      const size_t smem = (size_t)4 * 2 * words_per_cta(L, 4) * 4 + tab_bytes(4);
      int maxc = 0;
      if (cf && raise_smem_limit((const void *)cf, smem) ==
                    cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)cluster_ctas);
        cfg.blockDim = dim3(512u);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 4;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&maxc, (const void *)cf, &cfg) != cudaSuccess) maxc = 0;
      }
      cudaGetLastError();
      grid = maxc > 0 && cluster_ctas > 4 * maxc;
    }
    if (grid) p.S = 0;
  } else if (L == 32 && i8) {
    p.S = 2; p.G = 1; p.GT = 1; p.threads = 256;  // two z slabs per replica, one word per thread
  } else if (L == 16 && i8) {
    p.S = 1; p.G = 8; p.GT = 1; p.threads = 512;
  } else if (i8) {
    p.S = 1; p.G = 16; p.GT = 1; p.threads = 128;
  } else if (L == 32) {
    // four z slabs per replica, every word split over four warps (C3: 408 against 390 attempts/ns
    // for two slabs of one word per thread)
    p.S = 4; p.G = 1; p.GT = 1; p.threads = 512; p.NS = 4;
  } else if (L == 16) {
    p.S = 1; p.G = 4; p.GT = 1; p.threads = 512; p.NS = 4;  // C2: 23.3 against 16.7
  } else {
    p.S = 1; p.G = 4; p.GT = 1; p.threads = 512; p.NS = 4;  // C1: 3.1 against 1.5
  }
  // "S,G,GT,threads": the tuner's current candidate, else a tuned shape for this (L, R, field),
  // else the RFIM_BITS_PLAN environment override, else the defaults above
  std::string tuned;
  {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    auto it = g_tuned.find({L, Rcap, bimodal});
    if (it != g_tuned.end()) tuned = it->second;
  }
  const char *o = t_plan_override ? t_plan_override : (!tuned.empty() ? tuned.c_str() : getenv("RFIM_BITS_PLAN"));
  if (o) {
    int s, g, gt, th, ns = 1;
    // "S,G,GT,threads[,NS]" (NS = 4: every word split over four warps); an override that names no
    // instance for this L (e.g. an L=64 shape while building L=16) is ignored and the defaults stand
    const int nf = sscanf(o, "%d,%d,%d,%d,%d", &s, &g, &gt, &th, &ns);
    const bool named = nf == 4 || nf == 5;
    if (nf == 4) ns = 1;
    const bool exists = named && (s == 0 ? (ns == 1 && th >= 256 && th <= 1024 && th % 32 == 0 &&
                                            grid_kernel_for(L, g, gt, th, bimodal, i8))
                                         : kernel_for(L, s, gt, th, bimodal, i8, ns) != nullptr);
    if (exists) {
      p.S = s; p.G = g; p.GT = gt; p.threads = th; p.NS = ns;
    }
  }
  if (p.S != 0) {
    if (p.G > Rcap) p.G = Rcap;
    if (p.GT > p.G) p.GT = 1;
    if (p.G % p.GT) p.G = (p.G / p.GT) * p.GT;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  KernelFn fn = p.S == 0 ? nullptr : kernel_for(L, p.S, p.GT, p.threads, bimodal, i8, p.NS);
  GridFn gfn = p.S == 0 && p.threads >= 256 && p.threads <= 1024 ? grid_kernel_for(L, p.G, p.GT, p.threads, bimodal, i8) : nullptr;
  if (!fn && !gfn) {
    if (err) *err = "no bit-layout kernel instance for this plan";
    return -1;  // RFIM_EINVAL
  }
  if (gfn) {
    p.sms = sms;
    // largest partition over every R the context can reach
    int maxu = 0;
    for (int32_t R = 2; R <= Rcap; ++R) {
      BitsPlan q = p;
      maxu = std::max(maxu, grid_args(q, R, sms).max_units);
    }
    if (maxu > 255) {
      if (err) *err = "grid plan: too many planes per CTA";
      return -1;
    }
    p.smem = grid_smem(L, p.G, maxu, Rcap);
  }
  if (!gfn)
    p.smem = (size_t)p.G * 2 * words_per_cta(L, p.S) * 4 + tab_bytes(p.G);
  if (p.smem > 227 * 1024) {
    if (err) *err = "bit-layout plan exceeds shared memory";
    return -1;
  }
  const void *fptr = gfn ? (const void *)gfn : (const void *)fn;
  cudaError_t e = raise_smem_limit(fptr, p.smem);
  if (e == cudaSuccess && p.S > 1)
    e = cudaFuncSetAttribute(fptr, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) {
    if (err) *err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
    return -3;  // RFIM_ECUDA
  }
  auto grab = [&](void **ptr, size_t bytes, const char *what) -> int {
    cudaError_t ee = cudaMalloc(ptr, bytes);
    if (ee != cudaSuccess) {
      cudaGetLastError();
      *ptr = nullptr;
      if (err) *err = std::string("cudaMalloc(") + what + "): " + cudaGetErrorString(ee);
      return ee == cudaErrorMemoryAllocation ? -2 : -3;
    }
    return 0;
  };
  int rc = 0;
  if (!bimodal) {
    const int64_t W = (int64_t)L * L * L / 64, wpad = (W + 31) / 32 * 32;
    rc = grab((void **)&p.field4, sizeof(float4) * 2 * wpad * 8, "field4");
    if (!rc) rc = grab((void **)&p.flimb, sizeof(uint4) * 2 * 10 * wpad, "field limbs");
    if (!rc) rc = grab((void **)&p.fquant, sizeof(FieldQuant), "field quantum");
  }
  const size_t parts = (size_t)Rcap * p.S;
  if (!rc) rc = grab((void **)&p.partB, parts * 8, "partials");
  if (!rc) rc = grab((void **)&p.partM, parts * 8, "partials");
  if (!rc) rc = grab((void **)&p.partFi, parts * 8, "partials");
  if (!rc) rc = grab((void **)&p.partF, parts * 8, "partials");
  if (!rc) rc = grab((void **)&p.counter, 16, "counter");  // cluster arrivals, error word, grid-wide arrival count
  if (!rc && gfn) {
    const size_t gslots = 2 * (size_t)Rcap * (L + 1);  // two intervals' partials
    rc = grab((void **)&p.gpartB, gslots * 8, "grid partials");
    if (!rc) rc = grab((void **)&p.gpartM, gslots * 8, "grid partials");
    if (!rc) rc = grab((void **)&p.gpartFi, gslots * 8, "grid partials");
    if (!rc) rc = grab((void **)&p.gpartF, gslots * 8, "grid partials");
    if (!rc) rc = grab((void **)&p.prog, (size_t)std::max(sms, 1) * 4, "progress words");
    // int8 layout: the published end planes (halos) in the bit layout
    if (!rc && i8) rc = grab((void **)&p.gbits, (size_t)Rcap * 2 * ((size_t)L * L * L / 64) * 4, "halo words");
  }
  if (!rc && cudaMemset(p.counter, 0, 16) != cudaSuccess) rc = -3;
  if (!rc && p.prog && cudaMemset(p.prog, 0, (size_t)std::max(sms, 1) * 4) != cudaSuccess) rc = -3;
  if (rc) {
    free_bits_plan(p);
    return rc;
  }
  *plan = p;
  return 0;
}

bool bits_plan_fits(const BitsPlan &plan, int32_t R) { return R <= plan.Rcap; }

void free_bits_plan(BitsPlan &plan) {
  void *ptrs[] = {plan.field4, plan.flimb, plan.fquant, plan.partB, plan.partM, plan.partFi, plan.partF,
                  plan.counter, plan.gpartB, plan.gpartM, plan.gpartFi, plan.gpartF, plan.prog, plan.gbits};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  plan.field4 = nullptr;
  plan.flimb = nullptr;
  plan.fquant = nullptr;
  plan.partB = plan.partM = plan.partFi = nullptr;
  plan.partF = nullptr;
  plan.counter = nullptr;
  plan.gpartB = plan.gpartM = plan.gpartFi = nullptr;
  plan.gpartF = nullptr;
  plan.prog = nullptr;
  plan.gbits = nullptr;
}

cudaError_t build_field4(const RealView &v, BitsPlan &plan, cudaStream_t st) {
  if (!plan.field4) return cudaSuccess;
  const int64_t W = (int64_t)v.N / 64, wpad = (W + 31) / 32 * 32;
  k_build_field4<<<(int)((2 * W * 8 + 255) / 256), 256, 0, st>>>(v, plan.field4, wpad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !plan.flimb || !plan.fquant) return e;
  e = cudaMemsetAsync(plan.fquant, 0, sizeof(FieldQuant), st);
  if (e != cudaSuccess) return e;
  k_field_absmax<<<152, 256, 0, st>>>(v, &plan.fquant->fmax);
  k_field_limbs<<<(int)std::min<int64_t>((2 * W * 8 + 255) / 256, 4 * 152), 256, 0, st>>>(v, plan.flimb, plan.fquant, wpad);
  return cudaGetLastError();
}

cudaError_t launch_sweeps_bits(const RealView &v, const BitsPlan &plan, uint32_t sweep0, int32_t n_sweeps,
                               bool exchange, uint32_t j, int64_t measure_from, double J, double h,
                               cudaStream_t st, const MultiHit *mh, int32_t n_intervals) {
  ExchArgs xa{};
  xa.enabled = exchange ? 1 : 0;
  xa.j = j;
  xa.measure_from = measure_from;
  xa.J = J;
  xa.h = h;
  xa.partB = plan.partB;
  xa.partM = plan.partM;
  xa.partFi = plan.partFi;
  xa.partF = plan.partF;
  xa.counter = plan.counter;
  xa.expected = 0;  // set by the kernel to its grid size
  xa.ctl = nullptr;
  xa.err = plan.counter + 1;
  xa.flimb = plan.flimb;
  xa.fquant = plan.fquant;
  if (plan.S == 0) {
    GridFn gfn = grid_kernel_for(plan.L, plan.G, plan.GT, plan.threads, v.kind == kBimodal, plan.i8);
    if (!gfn || (plan.i8 && !plan.gbits)) return cudaErrorInvalidConfiguration;
    RealView vg = v;
    if (plan.i8) vg.bits = plan.gbits;  // halos go through the bit-layout scratch
    if (n_intervals < 1) return cudaErrorInvalidValue;
    GridArgs ga = grid_args(plan, v.R, plan.sms);
    const uint32_t niv = (uint32_t)(exchange ? n_intervals : 1);
    const uint32_t add = 2u * (uint32_t)n_sweeps * niv;
    const uint32_t arrivals = exchange ? (uint32_t)ga.gp.P * niv : 0u;  // one per CTA and interval
    if (plan.prog_base > 0xFFFFFFFFu - add) {  // the count would wrap: start again from zero
      const cudaError_t e = cudaMemsetAsync(plan.prog, 0, (size_t)plan.sms * 4, st);
      if (e != cudaSuccess) return e;
      plan.prog_base = 0;
    }
    if (plan.arrive_base > 0xFFFFFFFFu - arrivals) {
      const cudaError_t e = cudaMemsetAsync(plan.counter + 2, 0, 4, st);
      if (e != cudaSuccess) return e;
      plan.arrive_base = 0;
    }
    ga.prog_base = plan.prog_base;
    ga.n_iv = (int32_t)niv;
    ga.arrive_base = plan.arrive_base;
    plan.prog_base += add;
    plan.arrive_base += arrivals;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ga.gp.P);
    cfg.blockDim = dim3((unsigned)plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, gfn, vg, ga, sweep0, n_sweeps, (const float4 *)plan.field4, xa);
    if (le != cudaSuccess) {  // nothing ran: the words did not advance
      plan.prog_base -= add;
      plan.arrive_base -= arrivals;
    }
    return le;
  }
  if (n_intervals != 1) return cudaErrorInvalidValue;  // several intervals: grid-wide plan only
  const bool multihit = mh && mh->mh > 0;
  if (multihit && plan.S == 0) return cudaErrorInvalidConfiguration;
  KernelFn fn = multihit ? nullptr : kernel_for(plan.L, plan.S, plan.GT, plan.threads, v.kind == kBimodal, plan.i8, plan.NS);
  MhFn mfn = multihit ? mh_kernel_for(plan.L, plan.S, plan.GT, plan.threads, v.kind == kBimodal, mh->tile) : nullptr;
  if (!fn && !mfn) return cudaErrorInvalidConfiguration;
  const int clusters = (v.R + plan.G - 1) / plan.G;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * plan.S));
  cfg.blockDim = dim3((unsigned)plan.threads);
  cfg.dynamicSmemBytes = plan.smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  if (plan.S > 1) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)plan.S;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  if (mfn)
    return cudaLaunchKernelEx(&cfg, mfn, v, (int32_t)plan.G, sweep0, n_sweeps, (const float4 *)plan.field4, xa, *mh);
  return cudaLaunchKernelEx(&cfg, fn, v, (int32_t)plan.G, sweep0, n_sweeps, (const float4 *)plan.field4, xa);
}

}  // namespace rfim

// ---------------------------------------------------------------------------------------------
// Host self-check of the bit-layout neighbour words against direct neighbour lookup (no GPU).
namespace {

template <int L>
int selftest_bits_L(uint32_t seed) {
  using namespace rfim;
  using Gm = BitsGeom<L>;
  const int N = L * L * L, Lh = L / 2, W = Gm::W, P = Gm::P;
  std::vector<int> s(N);
  uint32_t x = seed | 1u;
  for (int i = 0; i < N; ++i) {
    x ^= x << 13; x ^= x >> 17; x ^= x << 5;
    s[i] = (x >> 7) & 1;
  }
  std::vector<uint32_t> bits(2 * W, 0u);
  for (int i = 0; i < N; ++i) {
    const int xx = i % L, yy = (i / L) % L, zz = i / (L * L);
    const int c = (xx + yy + zz) & 1;
    const int64_t q = q_of(L, Lh, xx, yy, zz);
    bits[c * W + (q >> 5)] |= (uint32_t)s[i] << bit_of(q);
  }
  int bad = 0;
  for (int c = 0; c < 2; ++c) {
    const uint32_t *O = bits.data() + (1 - c) * W;
    for (int wq = 0; wq < W; ++wq) {
      const int z = wq / P, iw = wq % P;
      uint32_t A, B, C, D;
      nb_xy<L>(O[z * P + iw], O[z * P + (iw + 1) % P], O[z * P + (iw + P - 1) % P], parity0_mask<L>(c, z, iw), A, B, C,
               D);
      const uint32_t E = O[((z + 1) % L) * P + iw], F = O[((z + L - 1) % L) * P + iw];
      uint32_t c0, c1, c2;
      count6(A, B, C, D, E, F, c0, c1, c2);
      for (int p = 0; p < 32; ++p) {
        const int64_t q = (int64_t)wq * 32 + p;
        const Site st = site_of_q(L, Lh, c, q);
        const int b = bit_of(q);
        auto at = [&](int xx, int yy, int zz) { return s[((zz + L) % L) * L * L + ((yy + L) % L) * L + (xx + L) % L]; };
        const int xm = at(st.x - 1, st.y, st.z), xp = at(st.x + 1, st.y, st.z);
        const int a = (A >> b) & 1, bb = (B >> b) & 1;
        const bool x_ok = (a + bb == xm + xp) && ((a == xm && bb == xp) || (a == xp && bb == xm));
        const bool y_ok = (int)((C >> b) & 1) == at(st.x, st.y + 1, st.z) && (int)((D >> b) & 1) == at(st.x, st.y - 1, st.z);
        const bool z_ok = (int)((E >> b) & 1) == at(st.x, st.y, st.z + 1) && (int)((F >> b) & 1) == at(st.x, st.y, st.z - 1);
        const int cnt = (int)(((c0 >> b) & 1) + 2 * ((c1 >> b) & 1) + 4 * ((c2 >> b) & 1));
        const int ref = xm + xp + at(st.x, st.y + 1, st.z) + at(st.x, st.y - 1, st.z) + at(st.x, st.y, st.z + 1) +
                        at(st.x, st.y, st.z - 1);
        if (!x_ok || !y_ok || !z_ok || cnt != ref) ++bad;
      }
    }
  }
  return bad;
}

}  // namespace

extern "C" int rfim_selftest_bits(int32_t L, uint32_t seed) {
  switch (L) {
    case 8: return selftest_bits_L<8>(seed);
    case 16: return selftest_bits_L<16>(seed);
    case 32: return selftest_bits_L<32>(seed);
    case 64: return selftest_bits_L<64>(seed);
    default: return -1;
  }
}

// Host self-check of the grid-wide partition: every unit has exactly one owner consistent with
// the CTA ranges, pieces tile each range inside single groups, at most kGridMaxPieces per CTA.
namespace {
// words[0]: progress word, words[1]: error word
__global__ void k_selftest_wait(unsigned *words, unsigned limit) {
  if (threadIdx.x == 0) rfim::grid_wait(words, 0, 1u, words + 1, limit);
}
}  // namespace

extern "C" int rfim_selftest_wait(int32_t spin_limit, int32_t set_flag) {
  if (spin_limit < 1 || spin_limit > (int32_t)rfim::kGridSpinLimit) return -1;  // RFIM_EINVAL
  unsigned *d = nullptr;
  unsigned h[2] = {set_flag ? 1u : 0u, 0u};
  if (cudaMalloc(&d, sizeof h) != cudaSuccess) return -3;  // RFIM_ECUDA
  cudaError_t e = cudaMemcpy(d, h, sizeof h, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_selftest_wait<<<1, 32>>>(d, (unsigned)spin_limit);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return -3;  // RFIM_ECUDA
  return h[1] ? -4 : 0;             // RFIM_ETIMEOUT : RFIM_OK
}

// Debug-build self-check of the check mechanism: a checked shared-memory index out of range is
// recorded in the error word and replaced by index 0, and the kernel finishes normally.
namespace {
__global__ void k_selftest_debug(unsigned *words, int index) {
  __shared__ unsigned cells[32];
  if (threadIdx.x < 32) cells[threadIdx.x] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    int i = index;
    if (!RFIM_DCHECK(words + 1, i >= 0 && i < 32, rfim::kDbgLattice)) i = 0;
    cells[i] = 7u;
  }
  __syncthreads();
  if (threadIdx.x == 0) words[0] = cells[0];
}
}  // namespace

extern "C" int rfim_debug_build(void) { return rfim::kDebugBuild ? 1 : 0; }

extern "C" int rfim_selftest_debug(void) {
  if (!rfim::kDebugBuild) return -6;  // RFIM_ESTATE: the checks are compiled only into librfim_debug.so
  unsigned *d = nullptr;
  unsigned h[2] = {0u, 0u};
  if (cudaMalloc(&d, sizeof h) != cudaSuccess) return -3;
  cudaError_t e = cudaMemcpy(d, h, sizeof h, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_selftest_debug<<<1, 32>>>(d, 40);  // out of range on purpose: the check must catch it
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return -3;
  return (h[0] == 7u && h[1] == rfim::kDbgLattice) ? 0 : -7;  // RFIM_OK : RFIM_EBOUNDS (not caught)
}

extern "C" int rfim_selftest_grid(int32_t L, int32_t R, int32_t P) {
  using namespace rfim;
  if (L < 2 || R < 2 || P < 1) return -1;
  GridPart gp{};
  gp.L = L;
  gp.NG = (R + kGridGroup - 1) / kGridGroup;
  gp.U = (int64_t)gp.NG * L;
  gp.P = P;
  int bad = 0;
  for (int k = 0; k < P; ++k) {
    const int64_t a = grid_begin(gp, k), b = grid_begin(gp, k + 1);
    for (int64_t u = a; u < b; ++u) bad += grid_owner(gp, u) != k;
    Piece pc[kGridMaxPieces];
    const int np = grid_pieces(gp, k, pc);
    int64_t covered = 0;
    for (int p = 0; p < np; ++p) {
      const int64_t u0 = (int64_t)pc[p].g * L + pc[p].z0;
      bad += u0 != a + pc[p].lu0;
      bad += pc[p].z0 + pc[p].n > L;
      bad += grid_slab_of(gp, k, pc[p].g) < 0;
      covered += pc[p].n;
    }
    bad += covered != b - a;
  }
  return bad;
}
