// Per-temperature tables computed on the host in double (compiled with -ffp-contract=off so every
// expression is rounded step by step, as in the plain definition).
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace rfim {

// Bimodal acceptance table for one temperature (computed in double on the host; this file is
// compiled with -ffp-contract=off so the expression is rounded step by step):
// dE = 2 (J s n + h s h_i), thr = floor(exp(-beta dE) 2^32) clamped to [1, 2^32 - 1] for dE > 0.
// Stored as thr - 1, and 0xFFFFFFFF for dE <= 0 (always accept).
void bimodal_row(double beta, float J, float h, uint32_t out[32]) {
  for (uint32_t idx = 0; idx < 32; ++idx) {
    const int32_t up = (int32_t)(idx & 7u);
    const int32_t si = (idx >> 3) & 1u ? 1 : -1;
    const int32_t fi = (idx >> 4) & 1u ? 1 : -1;
    if (up > 6) {
      out[idx] = 0u;
      continue;
    }
    const int32_t n = 2 * up - 6;
    const double dE = 2.0 * ((double)J * (double)(si * n) + (double)h * (double)(si * fi));
    if (dE <= 0.0) {
      out[idx] = 0xFFFFFFFFu;
      continue;
    }
    double p = std::floor(std::exp(-beta * dE) * 4294967296.0);
    if (p < 1.0) p = 1.0;
    if (p > 4294967295.0) p = 4294967295.0;
    out[idx] = (uint32_t)((uint64_t)p - 1u);
  }
}

void temperature_tables(const double *T, int32_t R, float J, float h, uint32_t *thr, float *b2, float *b2l,
                        double *beta, float gjn[8]) {
  for (int32_t k = 0; k < R; ++k) {
    beta[k] = 1.0 / T[k];
    b2[k] = 2.0f * (float)beta[k];
    b2l[k] = (float)(-1.4426950408889634 * (double)b2[k]);
    bimodal_row(beta[k], J, h, &thr[(size_t)k * 32]);
  }
  for (int u = 0; u < 8; ++u) gjn[u] = J * (float)(2 * u - 6);
}

void wave_tables(int32_t L, double *kcos, double *ksin) {
  const double K = 2.0 * 3.14159265358979323846 / (double)L;
  for (int32_t t = 0; t < L; ++t) {
    kcos[t] = std::cos(K * (double)t);
    ksin[t] = std::sin(K * (double)t);
  }
}

}  // namespace rfim
