// Throughput ceiling of the sweep's instruction mix on one SM, without lattice work: attempts per
// clock per SM for Philox4x32-10 alone and for Philox plus each acceptance test of the sweep
// kernels (decide.cuh; table entries addressed by a byte permute from a 256-byte aligned shared
// slot, as in kernels_bits.cuh).  One CTA per SM, 512 threads; each thread runs 8 blocks x 4
// replicas per iteration, with counters laid out as in the sweep (block index, replica, sweep,
// stream tag), so the compiler can share the same invariant products.  Cycles from clock64.
// Modes 3-5 are variants of the float-field test: the field of the block in registers (as in the
// sweep, instead of derived from a random word), the random word converted from a 64-bit
// integer, and tables holding two sites per 16-byte entry (one permute and one load per pair;
// the pair index is taken from random bits here, its formation from the bit slices not counted).
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "decide.cuh"
#include "philox.cuh"

using namespace rfim;

// MODE 0: Philox only, 1: + bimodal test, 2: + float-field test, 3: float test with the field in
// registers, 4: the same with a 64-bit-source conversion, 5: the same with two-site table entries
template <int MODE, int BAR>
__global__ void __launch_bounds__(512, 1) k_mix(uint32_t seed, int iters, uint32_t *out, unsigned long long *cyc) {
  __shared__ __align__(256) float2 tabf[64];
  __shared__ __align__(256) uint32_t tabu[128];
  __shared__ __align__(256) float4 tabp[256];  // two-site entries {b J n_a, b_a, b J n_b, b_b}
  for (int i = threadIdx.x; i < 64; i += blockDim.x) tabf[i] = make_float2(-2.0f + 0.25f * (i & 15), -0.7f);
  for (int i = threadIdx.x; i < 128; i += blockDim.x) tabu[i] = 0x40000000u + 977u * i;
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    tabp[i] = make_float4(-2.0f + 0.25f * (i & 15), -0.7f, -2.0f + 0.25f * (i >> 4), 0.7f);
  __syncthreads();
  const uint32_t slotp = (uint32_t)__cvta_generic_to_shared(tabp);
  float4 hh4[8];
#pragma unroll
  for (int j = 0; j < 8; ++j)
    hh4[j] = make_float4(0.3f * ((threadIdx.x + j) % 7) - 1.f, 0.1f * (j % 5) - 0.2f, 0.7f - 0.05f * j, 0.2f * (j % 3));
  const uint32_t slotf = (uint32_t)__cvta_generic_to_shared(tabf), slotu = (uint32_t)__cvta_generic_to_shared(tabu);
  uint32_t acc[4] = {0, 0, 0, 0}, fk[4] = {0, 0, 0, 0};
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    if (BAR > 0 && it % BAR == 0) __syncthreads();
#pragma unroll
    for (int jb = 0; jb < 8; ++jb) {
#pragma unroll
      for (int gg = 0; gg < 4; ++gg) {
        const Words4 w = philox10(seed, 7u, tid * 8u + jb, (uint32_t)gg, (uint32_t)it, 0x20000000u);
        if (MODE == 0) {
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] ^= w.w[q];
        } else if (MODE == 1) {
          const uint32_t offs = (w.w[0] ^ (uint32_t)(it * 0x9E3779B9u + gg)) & 0x7C7C7C7Cu;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t t;
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(t) : "r"(__byte_perm(offs, slotu, 0x7650u | q)));
            if (accept_table(w.w[q], t)) acc[gg] |= 1u << (8 * q + jb);
          }
        } else if (MODE == 2 || MODE == 3 || MODE == 4) {
          const uint32_t offs = (w.w[0] ^ (uint32_t)(it * 0x9E3779B9u + gg)) & 0x78787878u;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float2 e;
            asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(e.x), "=f"(e.y) : "r"(__byte_perm(offs, slotf, 0x7650u | q)));
            const float hr = q == 0 ? hh4[jb].x : q == 1 ? hh4[jb].y : q == 2 ? hh4[jb].z : hh4[jb].w;
            const float hh = MODE == 2 ? __uint_as_float(0x3f000000u | (w.w[(q + 1) & 3] >> 9)) : hr;
            if (MODE == 4) {
              const float wf = __ull2float_rz((unsigned long long)w.w[q]);
              const float r = __fmaf_rn(ex2_approx(__fmaf_rn(e.y, hh, e.x)), -4294967296.0f, wf);
              fk[q] = __funnelshift_l(__float_as_uint(r), fk[q], 1);
            } else {
              fk[q] = __funnelshift_l(accept_float_sign(w.w[q], e.x, hh, e.y), fk[q], 1);
            }
          }
        } else {
          const uint32_t po = (w.w[0] ^ (uint32_t)(it * 0x9E3779B9u + gg)) & 0x0FF00FF0u;
#pragma unroll
          for (int pr = 0; pr < 2; ++pr) {
            float4 e;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(e.x), "=f"(e.y), "=f"(e.z), "=f"(e.w)
                         : "r"(slotp + (pr ? (po >> 16) : (po & 0xFFFFu))));
            const float ha = pr ? hh4[jb].z : hh4[jb].x, hb = pr ? hh4[jb].w : hh4[jb].y;
            fk[2 * pr] = __funnelshift_l(accept_float_sign(w.w[2 * pr], e.x, ha, e.y), fk[2 * pr], 1);
            fk[2 * pr + 1] = __funnelshift_l(accept_float_sign(w.w[2 * pr + 1], e.z, hb, e.w), fk[2 * pr + 1], 1);
          }
        }
      }
    }
  }
  const unsigned long long t1 = clock64();
  out[tid] = acc[0] ^ acc[1] ^ acc[2] ^ acc[3] ^ fk[0] ^ fk[1] ^ fk[2] ^ fk[3];
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

template <int M, int B>
double rate(int sms, uint32_t *out, unsigned long long *cyc, unsigned long long *h) {
  const int threads = 512, iters = 200;
  for (int rep = 0; rep < 2; ++rep) k_mix<M, B><<<sms, threads>>>(1u, iters, out, cyc);
  if (cudaDeviceSynchronize() != cudaSuccess) return -1.0;
  cudaMemcpy(h, cyc, sms * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  unsigned long long mx = 0;
  for (int i = 0; i < sms; ++i) mx = h[i] > mx ? h[i] : mx;
  return (double)threads * iters * 8 * 4 * 4 / (double)mx;
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  uint32_t *out;
  unsigned long long *cyc;
  cudaMalloc(&out, (size_t)sms * 512 * 4);
  cudaMalloc(&cyc, sms * sizeof(unsigned long long));
  unsigned long long *h = new unsigned long long[sms];
  printf("attempts/clk/SM  Philox4x32-10 only:                  %.3f\n", rate<0, 0>(sms, out, cyc, h));
  printf("attempts/clk/SM  Philox + bimodal table test:         %.3f\n", rate<1, 0>(sms, out, cyc, h));
  printf("attempts/clk/SM  Philox + float-field test:           %.3f\n", rate<2, 0>(sms, out, cyc, h));
  printf("attempts/clk/SM  Philox + float-field test, barrier/2: %.3f\n", rate<2, 2>(sms, out, cyc, h));
  printf("attempts/clk/SM  float test, field in registers:       %.3f\n", rate<3, 0>(sms, out, cyc, h));
  printf("attempts/clk/SM  the same, 64-bit-source conversion:   %.3f\n", rate<4, 0>(sms, out, cyc, h));
  printf("attempts/clk/SM  the same, two-site table entries:     %.3f\n", rate<5, 0>(sms, out, cyc, h));
  delete[] h;
  cudaFree(out);
  cudaFree(cyc);
  return 0;
}
