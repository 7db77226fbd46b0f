// rfim_exchange_noalloc: the energy reduction and exchange step on caller-owned device buffers,
// with its scratch (per-(replica, slab) partial sums and the arrival counter) in a file-scope
// device array instead of memory the library allocates.  For callers that cannot allocate
// device memory: a framework or arena that owns all of it, or a latency-critical loop where
// cudaMalloc / cudaFree would synchronise the device.
//
// The array is shared by every call on a device and keeps the last call's contents; calls that
// overlap on the GPU (different streams, or host threads without ordering) race on it.  The
// arrival counter starts at zero (a file-scope device array is zero when the module loads) and
// the last CTA of each call sets it back to zero.
#include <algorithm>
#include <cstdint>
#include <string>

#include "rfim.h"
#include "bits_layout.cuh"
#include "debug_check.cuh"
#include "exchange.cuh"
#include "internal.h"
#include "lattice.cuh"

namespace rfim {

namespace {

// Scratch capacity: R * slabs partial slots.  4 x 8 bytes per slot plus the counter: 512 KiB + 256.
constexpr int kNoAllocSlots = 16384;
constexpr size_t kCounterOffset = (size_t)kNoAllocSlots * 32;
constexpr size_t kScratchBytes = kCounterOffset + 256;

static __device__ __align__(256) unsigned char g_exchange_scratch[kScratchBytes];

struct NoAllocArgs {
  RealView v;
  const float *field;  // unscaled h_i, natural order
  float h;
  double J;
  int32_t slabs;
};

template <typename T>
__device__ __forceinline__ T warp_add(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// One CTA per (replica, z slab): bond sum over the slab's colour-0 words (six neighbour words
// each, read from global memory), magnetisation and field term over all its words; then the
// last CTA adds the partials in slab order, forms E = -J B - F and takes exchange step j.
template <int L>
__global__ void __launch_bounds__(256) k_exchange_noalloc(NoAllocArgs a, uint32_t j, int64_t measure_from,
                                                          unsigned char *scratch) {
  using Gm = BitsGeom<L>;
  constexpr int P = Gm::P, W = Gm::W;
  const RealView &v = a.v;
  long long *partB = reinterpret_cast<long long *>(scratch);
  long long *partM = partB + kNoAllocSlots;
  long long *partFi = partM + kNoAllocSlots;
  double *partF = reinterpret_cast<double *>(partFi + kNoAllocSlots);
  unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + kCounterOffset);
  // debug build: this CTA's partial slot must lie inside the static array (else it writes none)
  const bool slot_ok = RFIM_DCHECK(counter + 1, blockIdx.x < (unsigned)kNoAllocSlots && gridDim.x <= (unsigned)kNoAllocSlots &&
                                                    (int)blockIdx.x / a.slabs < v.R,
                                   kDbgScratch);
  const int r = blockIdx.x / a.slabs, slab = blockIdx.x % a.slabs;
  const int z0 = (int)((int64_t)slab * L / a.slabs), z1 = (int)((int64_t)(slab + 1) * L / a.slabs);
  const uint32_t *S0 = v.bits + (int64_t)r * 2 * W, *S1 = S0 + W;
  long long b = 0, m = 0, fi = 0;
  float fs = 0.f, fe = 0.f;
  for (int t = threadIdx.x; t < 2 * (z1 - z0) * P; t += blockDim.x) {
    const int c = t / ((z1 - z0) * P), rem = t % ((z1 - z0) * P);
    const int z = z0 + rem / P, iw = rem % P;
    const int wq = z * P + iw;
    const uint32_t self = (c ? S1 : S0)[wq];
    m += 2 * __popc(self) - 32;
    if (c == 0) {
      const uint32_t *O = S1;
      uint32_t A, B, C, D;
      nb_xy<L>(O[wq], O[z * P + (iw + 1) % P], O[z * P + (iw + P - 1) % P], parity0_mask<L>(0, z, iw), A, B, C, D);
      const uint32_t E = O[((z + 1) % L) * P + iw], F = O[((z + L - 1) % L) * P + iw];
      b += 6 * 32 - 2 * (__popc(self ^ A) + __popc(self ^ B) + __popc(self ^ C) + __popc(self ^ D) + __popc(self ^ E) +
                         __popc(self ^ F));
    }
    for (int p = 0; p < 32; ++p) {
      const int64_t q = (int64_t)wq * 32 + p;
      const Site st = site_of_q(L, L / 2, c, q);
      const float hv = a.field[(int64_t)st.x + (int64_t)L * ((int64_t)st.y + (int64_t)L * st.z)];
      const bool up = (self >> bit_of(q)) & 1u;
      if (v.kind == kBimodal) {
        fi += (up == (hv > 0.0f)) ? 1 : -1;
      } else {
        const float hh = __fmul_rn(a.h, hv);
        const float term = up ? hh : -hh;
        const float tsum = __fadd_rn(fs, term);
        const float bp = __fsub_rn(tsum, fs);
        fe = __fadd_rn(fe, __fadd_rn(__fsub_rn(fs, __fsub_rn(tsum, bp)), __fsub_rn(term, bp)));
        fs = tsum;
      }
    }
  }
  __shared__ long long si[3][8];
  __shared__ double sd[8];
  __shared__ int last;
  b = warp_add(b);
  m = warp_add(m);
  fi = warp_add(fi);
  double fd = warp_add((double)fs + (double)fe);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    si[0][wid] = b;
    si[1][wid] = m;
    si[2][wid] = fi;
    sd[wid] = fd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tb = 0, tm = 0, tf = 0;
    double td = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tb += si[0][w];
      tm += si[1][w];
      tf += si[2][w];
      td += sd[w];
    }
    if (slot_ok) {
      partB[blockIdx.x] = tb;
      partM[blockIdx.x] = tm;
      partFi[blockIdx.x] = tf;
      partF[blockIdx.x] = td;
    }
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int rr = threadIdx.x; rr < v.R; rr += blockDim.x) {
    long long tb = 0, tm = 0, tf = 0;
    double td = 0.0;
    for (int q = 0; q < a.slabs; ++q) {
      const int64_t slot = (int64_t)rr * a.slabs + q;
      tb += __ldcg(partB + slot);
      tm += __ldcg(partM + slot);
      tf += __ldcg(partFi + slot);
      td += __ldcg(partF + slot);
    }
    const double Fv = v.kind == kBimodal ? (double)a.h * (double)tf : td;
    v.E[rr] = -a.J * (double)tb - Fv;
    v.M[rr] = tm;
  }
  __syncthreads();
  exchange_and_measure(v, j, measure_from);
  if (threadIdx.x == 0) *counter = 0u;
}

}  // namespace

}  // namespace rfim

using namespace rfim;

extern "C" int rfim_exchange_noalloc(const rfim_exchange_buffers *b, uint32_t j, int64_t measure_from, void *stream) {
  if (!b) return set_thread_error(RFIM_EINVAL, "rfim_exchange_noalloc: null buffers");
  const int32_t L = b->L, R = b->R;
  if (!(L == 8 || L == 16 || L == 32 || L == 64))
    return set_thread_error(RFIM_EINVAL, "rfim_exchange_noalloc: L must be 8, 16, 32 or 64");
  if (R < 2) return set_thread_error(RFIM_EINVAL, "rfim_exchange_noalloc: R must be >= 2");
  if (!b->spins || !b->field || !b->beta || !b->t2r || !b->r2t || !b->att || !b->acc || !b->obs || !b->n_meas || !b->E ||
      !b->M)
    return set_thread_error(RFIM_EINVAL, "rfim_exchange_noalloc: a buffer pointer is null");
  // z slabs per replica: enough CTAs to fill the GPU, bounded by the scratch capacity
  int slabs = std::max(1, std::min(L, 608 / R));
  if ((int64_t)R * slabs > kNoAllocSlots) slabs = kNoAllocSlots / R;
  if (slabs < 1)
    return set_thread_error(RFIM_EINVAL, "rfim_exchange_noalloc: R exceeds the static scratch capacity (16384 replicas)");
  cudaStream_t st = (cudaStream_t)stream;
  // In host code g_exchange_scratch names a host-side stand-in, not device memory: the kernel
  // gets the array's device address on the current device, looked up on every call (no stream
  // work; a cached address would go stale after cudaDeviceReset).
  unsigned char *scratch = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void **)&scratch, g_exchange_scratch);
  if (e != cudaSuccess || !scratch)
    return set_thread_error(RFIM_ECUDA, std::string("rfim_exchange_noalloc: cudaGetSymbolAddress: ") +
                                            cudaGetErrorString(e));
  NoAllocArgs a{};
  a.v.L = L;
  a.v.Lh = L / 2;
  a.v.N = L * L * L;
  a.v.R = R;
  a.v.kind = b->field_kind == RFIM_FIELD_BIMODAL ? kBimodal : kGaussian;
  a.v.seed = b->seed;
  a.v.realization = b->realization;
  a.v.stage = b->stage;
  a.v.bits = const_cast<uint32_t *>(b->spins);
  a.v.beta_d = b->beta;
  a.v.t2r = b->t2r;
  a.v.r2t = b->r2t;
  a.v.E = b->E;
  a.v.M = b->M;
  a.v.att = b->att;
  a.v.acc = b->acc;
  a.v.obs = b->obs;
  a.v.n_meas = b->n_meas;
  a.field = b->field;
  a.h = b->h;
  a.J = (double)b->J;
  a.slabs = slabs;
  const int grid = R * slabs;
  switch (L) {
    case 8: k_exchange_noalloc<8><<<grid, 256, 0, st>>>(a, j, measure_from, scratch); break;
    case 16: k_exchange_noalloc<16><<<grid, 256, 0, st>>>(a, j, measure_from, scratch); break;
    case 32: k_exchange_noalloc<32><<<grid, 256, 0, st>>>(a, j, measure_from, scratch); break;
    default: k_exchange_noalloc<64><<<grid, 256, 0, st>>>(a, j, measure_from, scratch); break;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_thread_error(RFIM_ECUDA, std::string("rfim_exchange_noalloc: launch: ") + cudaGetErrorString(e));
  if (kDebugBuild) {  // debug build only: wait for the launch and report its bounds checks
    unsigned int word = 0, zero = 0;
    unsigned int *err = reinterpret_cast<unsigned int *>(scratch + kCounterOffset) + 1;
    e = cudaMemcpyAsync(&word, err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && word) e = cudaMemcpyAsync(err, &zero, 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
      return set_thread_error(RFIM_ECUDA, std::string("rfim_exchange_noalloc: ") + cudaGetErrorString(e));
    if (word) return set_thread_error(RFIM_EBOUNDS, "rfim_exchange_noalloc: a bounds check of the debug build failed");
  }
  return RFIM_OK;
}
