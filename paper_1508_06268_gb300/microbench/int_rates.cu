// GB300 throughput microbenchmark: per-SM per-clock issue rates of the integer/float ops the
// sweep uses, Philox4x32-10 words per clock, L2 read bandwidth and cluster occupancy.  One CTA
// per SM, 1024 threads, in-bounds accesses only, no waits.  Built and run by bench.py --int-rates.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d: %s\n", #x, __LINE__, cudaGetErrorString(e)); return 1; } } while (0)

constexpr int ITERS = 2048;
constexpr int CH = 8;

__device__ __forceinline__ uint32_t lop3_x(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d; asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c)); return d;
}

template <int OP>
__global__ void k_op(uint32_t* out, long long* cyc, uint32_t seed) {
  uint32_t x[CH];
  float f[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) { x[c] = threadIdx.x * 7 + c + seed; f[c] = 0.001f * (threadIdx.x + c); }
  uint32_t a = seed ^ 0x1234567u, b = seed + 0x9e3779b9u;
  __syncthreads();
  long long t0 = clock64();
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (OP == 0) { x[c] = lop3_x(x[c], a, b); }
      else if (OP == 1) { asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(a), "r"(b)); }
      else if (OP == 2) { asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(x[c]) : "r"(a)); }
      else if (OP == 3) { uint64_t w; asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(w) : "r"(x[c]), "r"(a)); x[c] = (uint32_t)w ^ (uint32_t)(w >> 32); }
      else if (OP == 4) { asm volatile("add.u32 %0, %0, %1;" : "+r"(x[c]) : "r"(a)); }
      else if (OP == 5) { float g; asm volatile("cvt.rn.f32.u32 %0, %1;" : "=f"(g) : "r"(x[c])); x[c] = __float_as_uint(g); }
      else if (OP == 6) { asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(f[c])); }
      else if (OP == 7) { asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[c]) : "f"(1.0001f), "f"(0.5f)); }
      else if (OP == 8) { asm volatile("add.f32 %0, %0, %1;" : "+f"(f[c]) : "f"(0.5f)); }
      else if (OP == 9) { uint32_t y; asm volatile("shf.l.wrap.b32 %0, %1, %1, 3;" : "=r"(y) : "r"(x[c])); x[c] = y; }
      else if (OP == 10) { uint32_t y; asm volatile("prmt.b32 %0, %1, %2, 0x3210;" : "=r"(y) : "r"(x[c]), "r"(a)); x[c] = y ^ 1; }
    }
  }
  long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) acc ^= x[c] ^ __float_as_uint(f[c]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0, uint32_t k1) {
  uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
  uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
  uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
  c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
}

__global__ void k_philox(uint32_t* out, long long* cyc, uint32_t k0, uint32_t k1, int n) {
  uint32_t acc = 0;
  __syncthreads();
  long long t0 = clock64();
  for (int i = 0; i < n; ++i) {
    uint32_t c0 = threadIdx.x + i * 1024, c1 = blockIdx.x, c2 = 17, c3 = 0x20000000u;
    uint32_t a = k0, b = k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) { philox_round(c0, c1, c2, c3, a, b); a += 0x9E3779B9u; b += 0xBB67AE85u; }
    acc += c0 ^ c1 ^ c2 ^ c3;
  }
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void k_l2read(const uint4* __restrict__ buf, size_t n_vec, int reps, uint32_t* out, long long* cyc) {
  uint32_t acc = 0;
  __syncthreads();
  long long t0 = clock64();
  for (int r = 0; r < reps; ++r) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x + (size_t)r * 4096; i < n_vec + (size_t)r * 4096; i += (size_t)gridDim.x * blockDim.x) {
      uint4 v = __ldcg(buf + (i % n_vec));
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

int main() {
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, 0));
  int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("device %s sms=%d cc=%d.%d l2=%d smem/sm=%zu smem/blk_optin=%zu clock_khz=%d regs/sm=%d\n", p.name, p.multiProcessorCount, p.major, p.minor,
         p.l2CacheSize, p.sharedMemPerMultiprocessor, p.sharedMemPerBlockOptin, clk, p.regsPerMultiprocessor);
  const int SM = p.multiProcessorCount, T = 1024;
  uint32_t* out; long long* cyc; CK(cudaMalloc(&out, sizeof(uint32_t) * SM * T)); CK(cudaMalloc(&cyc, sizeof(long long) * SM));
  long long hc[1024];
  const char* names[] = {"LOP3", "IMAD(mad.lo)", "IMAD.HI(mul.hi)", "mul.wide+xor", "IADD", "I2F", "EX2", "FFMA", "FADD", "SHF", "PRMT+xor"};
  auto report = [&](const char* nm, double ops_per_thread) {
    cudaMemcpy(hc, cyc, sizeof(long long) * SM, cudaMemcpyDeviceToHost);
    double mx = 0, sum = 0; for (int i = 0; i < SM; ++i) { sum += hc[i]; if (hc[i] > mx) mx = hc[i]; }
    printf("%-18s %8.2f thread-ops/clk/SM (avg cycles %.0f)\n", nm, ops_per_thread * T / (sum / SM), sum / SM);
  };
#define RUN(OPN) do { k_op<OPN><<<SM, T>>>(out, cyc, 1u); CK(cudaDeviceSynchronize()); k_op<OPN><<<SM, T>>>(out, cyc, 2u); CK(cudaDeviceSynchronize()); report(names[OPN], (double)ITERS * CH); } while (0)
  RUN(0); RUN(1); RUN(2); RUN(3); RUN(4); RUN(5); RUN(6); RUN(7); RUN(8); RUN(9); RUN(10);
  {
    int n = 256;
    k_philox<<<SM, T>>>(out, cyc, 42u, 7u, n); CK(cudaDeviceSynchronize());
    k_philox<<<SM, T>>>(out, cyc, 42u, 7u, n); CK(cudaDeviceSynchronize());
    cudaMemcpy(hc, cyc, sizeof(long long) * SM, cudaMemcpyDeviceToHost);
    double sum = 0; for (int i = 0; i < SM; ++i) sum += hc[i];
    double calls_per_clk = (double)n * T / (sum / SM);
    printf("Philox4x32-10      %8.3f calls/clk/SM  -> words/clk/SM %.2f\n", calls_per_clk, 4 * calls_per_clk);
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    cudaEventRecord(e0); k_philox<<<SM, T>>>(out, cyc, 42u, 7u, 4096); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    printf("Philox4x32-10      %8.1f Gwords/s (events, n=4096)\n", 4.0 * 4096 * T * SM / (ms * 1e6));
  }
  for (size_t mb : {1, 8, 32, 64}) {
    size_t bytes = mb << 20, nv = bytes / 16;
    uint4* buf; CK(cudaMalloc(&buf, bytes)); CK(cudaMemset(buf, 1, bytes));
    int reps = (int)(2048 / mb);
    k_l2read<<<SM, T>>>(buf, nv, 2, out, cyc); CK(cudaDeviceSynchronize());
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    cudaEventRecord(e0); k_l2read<<<SM, T>>>(buf, nv, reps, out, cyc); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    cudaMemcpy(hc, cyc, sizeof(long long) * SM, cudaMemcpyDeviceToHost);
    double sum = 0; for (int i = 0; i < SM; ++i) sum += hc[i];
    double tot = (double)bytes * reps;
    printf("L2 read %3zu MB: %8.1f GB/s (events)  %6.1f B/clk/SM\n", mb, tot / (ms * 1e6), tot / SM / (sum / SM));
    cudaFree(buf);
  }
  // cluster occupancy with ~100 KB and ~200 KB smem per CTA
  for (int smem : {40 * 1024, 100 * 1024, 200 * 1024}) {
    for (int cs : {1, 2, 4, 8, 16}) {
      cudaLaunchConfig_t cfg = {}; cudaLaunchAttribute at[1];
      cfg.gridDim = dim3(cs * 64); cfg.blockDim = dim3(1024); cfg.dynamicSmemBytes = smem;
      at[0].id = cudaLaunchAttributeClusterDimension; at[0].val.clusterDim.x = cs; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
      cfg.attrs = at; cfg.numAttrs = 1;
      cudaFuncSetAttribute(k_l2read, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (cs > 8) cudaFuncSetAttribute(k_l2read, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      int ncl = -1; cudaError_t e = cudaOccupancyMaxActiveClusters(&ncl, (void*)k_l2read, &cfg);
      printf("smem %6d cluster %2d: max active clusters %d (%s) -> CTAs %d\n", smem, cs, ncl, cudaGetErrorString(e), ncl * cs);
      cudaGetLastError();
    }
  }
  return 0;
}
