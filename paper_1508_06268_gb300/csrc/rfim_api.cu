// Host side of the C ABI declared in include/rfim.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <numeric>
#include <queue>
#include <string>
#include <utility>
#include <vector>

#include "rfim.h"
#include "internal.h"
#include "sweep_bits.h"
#include "debug_check.cuh"

using namespace rfim;

struct rfim_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int32_t L = 0, Lh = 0, N = 0, R = 0, Rcap = 0;
  float J = 1.0f, h = 1.0f;
  int32_t kind = 0, layout = 0;
  uint32_t field_seed = 0, seed = 0, realization = 0, stage = 0;
  std::vector<double> T;
  int64_t sweep = 0, xstep = 0;
  int64_t launches = 0;
  // device buffers
  uint8_t *spins8 = nullptr;
  uint32_t *bits = nullptr;
  float *hraw = nullptr, *hh_c = nullptr;
  uint8_t *hbit_c = nullptr;
  uint32_t *hbits = nullptr;
  uint32_t *thr = nullptr;
  float *gjn = nullptr, *b2 = nullptr, *b2l = nullptr;
  double *beta_d = nullptr;
  int32_t *t2r = nullptr, *r2t = nullptr;
  double *E = nullptr;
  int64_t *M = nullptr;
  uint64_t *att = nullptr, *acc = nullptr;
  double *obs = nullptr;
  int64_t *n_meas = nullptr;
  int8_t *scratch8 = nullptr;  // int8[Rcap][N] staging for state conversion
  EnergyParts eparts{};        // int8 layout: partials of the multi-CTA energy reduction
  // structure-factor measurement (correlation length, Sec. 7): off unless enabled
  bool xi_on = false;
  double *sumF = nullptr, *kcos = nullptr, *ksin = nullptr;
  BitsPlan plan;
  MultiHit mh;  // multi-hit double checkerboard (mh.mh == 0: plain checkerboard)
  std::string err;
  // optional kernel timing: event pairs around sweep launches (kind 0) and energy+exchange (kind 1)
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used[2], ev_free;
  int64_t prof_units[2] = {0, 0};  // bracketed groups (a launch of K exchange intervals counts K)
};

namespace {

thread_local std::string g_create_error;

int fail(rfim_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx)
    ctx->err = buf;
  else
    g_create_error = buf;
  return code;
}

#define CUDA_OR_FAIL(ctx, call)                                                                            \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess)                                                                                 \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? RFIM_ENOMEM : RFIM_ECUDA, "%s: %s (%s:%d)", #call, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                                             \
  } while (0)

RealView view_of(const rfim_ctx *c) {
  RealView v;
  v.L = c->L;
  v.Lh = c->Lh;
  v.N = c->N;
  v.R = c->R;
  v.kind = c->kind;
  v.seed = c->seed;
  v.realization = c->realization;
  v.stage = c->stage;
  v.spins8 = c->spins8;
  v.bits = c->bits;
  v.hh_c = c->hh_c;
  v.hbit_c = c->hbit_c;
  v.hbits = c->hbits;
  v.thr = c->thr;
  v.gjn = c->gjn;
  v.b2 = c->b2;
  v.b2l = c->b2l;
  v.beta_d = c->beta_d;
  v.t2r = c->t2r;
  v.r2t = c->r2t;
  v.E = c->E;
  v.M = c->M;
  v.att = c->att;
  v.acc = c->acc;
  v.obs = c->obs;
  v.n_meas = c->n_meas;
  return v;
}

cudaError_t prof_begin(rfim_ctx *c, int kind, cudaEvent_t *stop_out, int64_t units = 1) {
  *stop_out = nullptr;
  if (!c->profiling) return cudaSuccess;
  c->prof_units[kind] += units;
  std::pair<cudaEvent_t, cudaEvent_t> ev;
  if (!c->ev_free.empty()) {
    ev = c->ev_free.back();
    c->ev_free.pop_back();
  } else {
    cudaError_t e = cudaEventCreate(&ev.first);
    if (e == cudaSuccess) e = cudaEventCreate(&ev.second);
    if (e != cudaSuccess) return e;
  }
  c->ev_used[kind].push_back(ev);
  *stop_out = ev.second;
  return cudaEventRecord(ev.first, c->stream);
}

cudaError_t prof_end(rfim_ctx *c, cudaEvent_t stop) {
  return stop ? cudaEventRecord(stop, c->stream) : cudaSuccess;
}

void free_events(rfim_ctx *c) {
  for (auto &v : c->ev_used)
    for (auto &p : v) c->ev_free.push_back(p);
  for (auto &v : c->ev_used) v.clear();
  for (auto &p : c->ev_free) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  c->ev_free.clear();
}

void free_all(rfim_ctx *c) {
  free_events(c);
  void *ptrs[] = {c->spins8, c->bits, c->hraw, c->hh_c, c->hbit_c, c->hbits, c->thr, c->gjn, c->b2, c->b2l,
                  c->beta_d, c->t2r, c->r2t, c->E, c->M, c->att, c->acc, c->obs, c->n_meas, c->scratch8,
                  c->sumF, c->kcos, c->ksin, c->eparts.B, c->eparts.M, c->eparts.Fi, c->eparts.F,
                  c->eparts.count};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  free_bits_plan(c->plan);
}

int upload_temps(rfim_ctx *c) {
  const int32_t R = c->R;
  std::vector<uint32_t> thr((size_t)R * 32);
  std::vector<float> b2(R), b2l(R);
  std::vector<double> beta(R);
  float gjn[8];
  temperature_tables(c->T.data(), R, c->J, c->h, thr.data(), b2.data(), b2l.data(), beta.data(), gjn);
  CUDA_OR_FAIL(c, cudaMemcpyAsync(c->thr, thr.data(), thr.size() * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_OR_FAIL(c, cudaMemcpyAsync(c->b2, b2.data(), R * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_OR_FAIL(c, cudaMemcpyAsync(c->b2l, b2l.data(), R * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_OR_FAIL(c, cudaMemcpyAsync(c->beta_d, beta.data(), R * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_OR_FAIL(c, cudaMemcpyAsync(c->gjn, gjn, sizeof gjn, cudaMemcpyHostToDevice, c->stream));
  // pageable sources: make sure the copies have consumed the host vectors before they go away
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  return RFIM_OK;
}

// Fresh random start at `stage` with identity permutation; counters and accumulators zero.
int reset_state(rfim_ctx *c, uint32_t stage) {
  c->stage = stage;
  c->sweep = 0;
  c->xstep = 0;
  RealView v = view_of(c);
  CUDA_OR_FAIL(c, launch_init_spins(v, c->R, stage, c->layout == RFIM_LAYOUT_BITPACK, c->stream));
  c->launches += 1;
  std::vector<int32_t> id(c->Rcap);
  std::iota(id.begin(), id.end(), 0);
  CUDA_OR_FAIL(c, cudaMemcpyAsync(c->t2r, id.data(), c->Rcap * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_OR_FAIL(c, cudaMemcpyAsync(c->r2t, id.data(), c->Rcap * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_OR_FAIL(c, cudaMemsetAsync(c->att, 0, c->Rcap * 8, c->stream));
  CUDA_OR_FAIL(c, cudaMemsetAsync(c->acc, 0, c->Rcap * 8, c->stream));
  CUDA_OR_FAIL(c, cudaMemsetAsync(c->obs, 0, (size_t)c->Rcap * 5 * 8, c->stream));
  if (c->sumF) CUDA_OR_FAIL(c, cudaMemsetAsync(c->sumF, 0, (size_t)c->Rcap * 8, c->stream));
  CUDA_OR_FAIL(c, cudaMemsetAsync(c->n_meas, 0, 8, c->stream));
  CUDA_OR_FAIL(c, cudaMemsetAsync(c->E, 0, c->Rcap * 8, c->stream));
  CUDA_OR_FAIL(c, cudaMemsetAsync(c->M, 0, c->Rcap * 8, c->stream));
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  return RFIM_OK;
}

// Bounded device waits that expired (bit-layout kernels) surface as RFIM_ETIMEOUT, failed bounds
// checks of the debug build as RFIM_EBOUNDS; the word is cleared once reported.  Synchronises the
// stream.
int check_device_error(rfim_ctx *c) {
  if (!c->plan.counter) return RFIM_OK;  // no bit-layout plan (int8 kernels of other L)
  unsigned int word = 0;
  CUDA_OR_FAIL(c, cudaMemcpyAsync(&word, c->plan.counter + 1, 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  if (!word) return RFIM_OK;
  CUDA_OR_FAIL(c, cudaMemsetAsync(c->plan.counter + 1, 0, 4, c->stream));
  if (c->plan.prog) {  // an expired wait can leave the grid-wide kernel's progress words uneven
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->plan.prog, 0, (size_t)std::max(c->plan.sms, 1) * 4, c->stream));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->plan.counter + 2, 0, 4, c->stream));
    c->plan.prog_base = 0;
    c->plan.arrive_base = 0;
  }
  if (word & kDbgMask)
    return fail(c, RFIM_EBOUNDS, "a bounds check of the debug build failed (error word 0x%x); the checked accesses were skipped", word);
  return fail(c, RFIM_ETIMEOUT, "a bounded device wait expired (error word %u); results of that launch are invalid", word);
}

int do_sweeps(rfim_ctx *c, int64_t n) {
  if (n <= 0) return RFIM_OK;
  RealView v = view_of(c);
  cudaEvent_t stop;
  CUDA_OR_FAIL(c, prof_begin(c, 0, &stop));
  if (c->plan.counter) {  // bit layout, or the int8 layout staged as bits
    CUDA_OR_FAIL(c, launch_sweeps_bits(v, c->plan, (uint32_t)c->sweep, (int32_t)n, false, 0u, 0, (double)c->J,
                                       (double)c->h, c->stream, &c->mh));
    c->launches += 1;
    c->sweep += n;
  } else {
    for (int64_t t = 0; t < n; ++t) {
      for (int colour = 0; colour < 2; ++colour) {
        CUDA_OR_FAIL(c, launch_halfsweep_int8(v, colour, (uint32_t)c->sweep, c->stream));
        c->launches += 1;
      }
      c->sweep += 1;
    }
  }
  CUDA_OR_FAIL(c, prof_end(c, stop));
  return RFIM_OK;
}

// After exchange step j: the structure factor of every replica when that step measured.
int measure_xi_after(rfim_ctx *c, int64_t j, int64_t measure_from) {
  if (!c->xi_on || j < measure_from) return RFIM_OK;
  CUDA_OR_FAIL(c, launch_measure_xi(view_of(c), c->kcos, c->ksin, c->sumF, c->layout == RFIM_LAYOUT_BITPACK, c->stream));
  c->launches += 1;
  return RFIM_OK;
}

// Bit layout: n sweeps and the exchange step in one launch (fused tail); with the grid-wide plan,
// k such intervals in one launch.
int do_sweeps_exchange_bits(rfim_ctx *c, int64_t n, int64_t measure_from, int32_t k = 1) {
  RealView v = view_of(c);
  cudaEvent_t stop;
  CUDA_OR_FAIL(c, prof_begin(c, 0, &stop, k));
  CUDA_OR_FAIL(c, launch_sweeps_bits(v, c->plan, (uint32_t)c->sweep, (int32_t)n, true, (uint32_t)c->xstep,
                                     measure_from, (double)c->J, (double)c->h, c->stream, &c->mh, k));
  CUDA_OR_FAIL(c, prof_end(c, stop));
  c->launches += 1;
  c->sweep += n * k;
  c->xstep += k;
  return measure_xi_after(c, c->xstep - 1, measure_from);
}

// Exchange intervals one grid-wide launch takes at most (the host regains control between them).
constexpr int64_t kMaxIntervalsPerLaunch = 64;

int do_exchange(rfim_ctx *c, int64_t measure_from) {
  if (c->plan.counter) return do_sweeps_exchange_bits(c, 0, measure_from);
  RealView v = view_of(c);
  cudaEvent_t stop;
  CUDA_OR_FAIL(c, prof_begin(c, 1, &stop));
  CUDA_OR_FAIL(c, launch_energy(v, (double)c->J, (double)c->h, c->layout == RFIM_LAYOUT_BITPACK, c->stream,
                                 c->eparts.count ? &c->eparts : nullptr));
  CUDA_OR_FAIL(c, launch_exchange(v, (uint32_t)c->xstep, measure_from, c->stream));
  CUDA_OR_FAIL(c, prof_end(c, stop));
  c->launches += 2;
  c->xstep += 1;
  return measure_xi_after(c, c->xstep - 1, measure_from);
}

int do_run(rfim_ctx *c, int64_t n_sweeps, int32_t ex, int64_t measure_from) {
  int64_t left = n_sweeps;
  while (left > 0) {
    int64_t chunk = left;
    if (ex > 0) {
      const int64_t to_next = ex - (c->sweep % ex);
      chunk = std::min(left, to_next);
    }
    const bool ends_interval = ex > 0 && (c->sweep + chunk) % ex == 0;
    int rc;
    // whole intervals on the grid-wide plan: several per launch (not with the structure factor,
    // which a separate kernel measures after every exchange step, nor with multi-hit)
    if (ends_interval && chunk == ex && left >= 2 * (int64_t)ex && c->plan.counter && c->plan.S == 0 &&
        !c->xi_on && c->mh.mh == 0) {
      const int64_t k = std::min(left / ex, kMaxIntervalsPerLaunch);
      rc = do_sweeps_exchange_bits(c, ex, measure_from, (int32_t)k);
      if (rc) return rc;
      left -= k * ex;
      continue;
    }
    if (ends_interval && c->plan.counter) {
      rc = do_sweeps_exchange_bits(c, chunk, measure_from);
      if (rc) return rc;
      left -= chunk;
      continue;
    }
    rc = do_sweeps(c, chunk);
    if (rc) return rc;
    left -= chunk;
    if (ends_interval) {
      rc = do_exchange(c, measure_from);
      if (rc) return rc;
    }
  }
  return RFIM_OK;
}

template <typename T>
int dalloc(rfim_ctx *c, T **p, size_t count) {
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T) > 0 ? count * sizeof(T) : 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, e == cudaErrorMemoryAllocation ? RFIM_ENOMEM : RFIM_ECUDA, "cudaMalloc(%zu bytes): %s",
                count * sizeof(T), cudaGetErrorString(e));
  }
  return RFIM_OK;
}

}  // namespace

int rfim::set_thread_error(int code, const std::string &msg) {
  g_create_error = msg;
  return code;
}

extern "C" {

int rfim_create(const rfim_config *cfg, rfim_ctx **out) {
  if (!cfg || !out) return fail(nullptr, RFIM_EINVAL, "null argument");
  *out = nullptr;
  const int32_t L = cfg->L, R = cfg->R, Rcap = cfg->R_capacity;
  if (L < 2 || (L & 1)) return fail(nullptr, RFIM_EINVAL, "L must be even and >= 2 (got %d)", L);
  if (L > 1024) return fail(nullptr, RFIM_EINVAL, "L too large (%d)", L);
  if (R < 2) return fail(nullptr, RFIM_EINVAL, "R must be >= 2 (got %d)", R);
  if (Rcap < R) return fail(nullptr, RFIM_EINVAL, "R_capacity (%d) < R (%d)", Rcap, R);
  if (Rcap > 65536) return fail(nullptr, RFIM_EINVAL, "R_capacity too large (%d)", Rcap);
  if (cfg->field_kind < 0 || cfg->field_kind > 2) return fail(nullptr, RFIM_EINVAL, "unknown field kind");
  if (cfg->field_kind == RFIM_FIELD_EXPLICIT && !cfg->field)
    return fail(nullptr, RFIM_EINVAL, "explicit field needs a field array");
  if (cfg->layout != RFIM_LAYOUT_INT8 && cfg->layout != RFIM_LAYOUT_BITPACK)
    return fail(nullptr, RFIM_EINVAL, "unknown layout");
  if (!cfg->temps) return fail(nullptr, RFIM_EINVAL, "temps is null");
  for (int32_t k = 0; k < R; ++k) {
    if (!(cfg->temps[k] > 0.0) || !std::isfinite(cfg->temps[k]))
      return fail(nullptr, RFIM_EINVAL, "temperature %d not positive", k);
    if (k > 0 && !(cfg->temps[k] > cfg->temps[k - 1]))
      return fail(nullptr, RFIM_EINVAL, "temperatures must be strictly ascending");
  }
  if (cfg->layout == RFIM_LAYOUT_BITPACK && !bits_supported(L))
    return fail(nullptr, RFIM_EINVAL, "bit layout supports L in {8,16,32,64} (got %d)", L);

  rfim_ctx *c = new rfim_ctx();
  cudaGetDevice(&c->device);
  c->stream = (cudaStream_t)cfg->stream;
  c->L = L;
  c->Lh = L / 2;
  c->N = L * L * L;
  c->R = R;
  c->Rcap = Rcap;
  c->J = cfg->J;
  c->h = cfg->h;
  c->kind = cfg->field_kind;
  c->layout = cfg->layout;
  c->field_seed = cfg->field_seed;
  c->seed = cfg->seed;
  c->realization = cfg->realization;
  c->T.assign(cfg->temps, cfg->temps + R);
  const size_t N = (size_t)c->N, half = N / 2;
  int rc = RFIM_OK;
  auto bail = [&](int code) {
    g_create_error = c->err;
    free_all(c);
    delete c;
    return code;
  };
  // int8 layout with L in {8, 16, 32, 64}: stored as bytes, swept by the bit-layout kernels that
  // stage each slab as bits in shared memory (kernels_bits_i8.cu)
  const bool staged_i8 = cfg->layout == RFIM_LAYOUT_INT8 && bits_supported(L);
  if (c->layout == RFIM_LAYOUT_BITPACK) {
    if ((rc = dalloc(c, &c->bits, (size_t)Rcap * N / 32))) return bail(rc);
    if ((rc = dalloc(c, &c->hbits, N / 32))) return bail(rc);
  } else {
    if (staged_i8 && (rc = dalloc(c, &c->hbits, N / 32))) return bail(rc);
    if ((rc = dalloc(c, &c->spins8, (size_t)Rcap * N))) return bail(rc);
    const size_t parts = (size_t)Rcap * kEnergyMaxParts;
    if ((rc = dalloc(c, &c->eparts.B, parts))) return bail(rc);
    if ((rc = dalloc(c, &c->eparts.M, parts))) return bail(rc);
    if ((rc = dalloc(c, &c->eparts.Fi, parts))) return bail(rc);
    if ((rc = dalloc(c, &c->eparts.F, parts))) return bail(rc);
    if ((rc = dalloc(c, &c->eparts.count, (size_t)Rcap))) return bail(rc);
    const cudaError_t e = cudaMemsetAsync(c->eparts.count, 0, (size_t)Rcap * 4, c->stream);
    if (e != cudaSuccess) return bail(fail(c, RFIM_ECUDA, "memset: %s", cudaGetErrorString(e)));
  }
  if ((rc = dalloc(c, &c->hraw, N))) return bail(rc);
  if ((rc = dalloc(c, &c->hh_c, N))) return bail(rc);
  if ((rc = dalloc(c, &c->hbit_c, N))) return bail(rc);
  if ((rc = dalloc(c, &c->thr, (size_t)Rcap * 32))) return bail(rc);
  if ((rc = dalloc(c, &c->gjn, 8))) return bail(rc);
  if ((rc = dalloc(c, &c->b2, Rcap))) return bail(rc);
  if ((rc = dalloc(c, &c->b2l, Rcap))) return bail(rc);
  if ((rc = dalloc(c, &c->beta_d, Rcap))) return bail(rc);
  if ((rc = dalloc(c, &c->t2r, Rcap))) return bail(rc);
  if ((rc = dalloc(c, &c->r2t, Rcap))) return bail(rc);
  if ((rc = dalloc(c, &c->E, Rcap))) return bail(rc);
  if ((rc = dalloc(c, &c->M, Rcap))) return bail(rc);
  if ((rc = dalloc(c, &c->att, Rcap))) return bail(rc);
  if ((rc = dalloc(c, &c->acc, Rcap))) return bail(rc);
  if ((rc = dalloc(c, &c->obs, (size_t)Rcap * 5))) return bail(rc);
  if ((rc = dalloc(c, &c->n_meas, 1))) return bail(rc);
  (void)half;
  if (c->layout == RFIM_LAYOUT_BITPACK || staged_i8) {
    if ((rc = make_bits_plan(L, Rcap, c->kind == kBimodal, &c->plan, &c->err, staged_i8))) return bail(rc);
  }
  if (c->kind == RFIM_FIELD_EXPLICIT) {
    cudaError_t e = cudaMemcpyAsync(c->hraw, cfg->field, N * 4, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return bail(fail(c, RFIM_ECUDA, "field upload: %s", cudaGetErrorString(e)));
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(fail(c, RFIM_ECUDA, "field upload: %s", cudaGetErrorString(e)));
  }
  {
    RealView v = view_of(c);
    cudaError_t e = launch_field(v, c->kind, c->field_seed, c->h, c->hraw, c->hh_c, c->hbit_c, c->hbits, c->stream);
    if (e != cudaSuccess) return bail(fail(c, RFIM_ECUDA, "field kernel: %s", cudaGetErrorString(e)));
    c->launches += c->hbits ? 2 : 1;
    if (c->plan.field4) {
      e = build_field4(v, c->plan, c->stream);
      if (e != cudaSuccess) return bail(fail(c, RFIM_ECUDA, "field4 kernel: %s", cudaGetErrorString(e)));
      c->launches += 1;
    }
  }
  if ((rc = upload_temps(c))) return bail(rc);
  if ((rc = reset_state(c, 0))) return bail(rc);
  *out = c;
  return RFIM_OK;
}

int rfim_destroy(rfim_ctx *ctx) {
  if (!ctx) return RFIM_OK;
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
  return RFIM_OK;
}

int rfim_sweep(rfim_ctx *ctx, int64_t n_sweeps) {
  if (!ctx) return RFIM_EINVAL;
  if (n_sweeps < 0) return fail(ctx, RFIM_EINVAL, "n_sweeps < 0");
  return do_sweeps(ctx, n_sweeps);
}

int rfim_exchange(rfim_ctx *ctx, int64_t measure_from) {
  if (!ctx) return RFIM_EINVAL;
  return do_exchange(ctx, measure_from);
}

int rfim_run(rfim_ctx *ctx, int64_t n_sweeps, int32_t exchange_every, int64_t measure_from) {
  if (!ctx) return RFIM_EINVAL;
  if (n_sweeps < 0) return fail(ctx, RFIM_EINVAL, "n_sweeps < 0");
  return do_run(ctx, n_sweeps, exchange_every, measure_from);
}

int rfim_adapt_temps(rfim_ctx *ctx, int32_t n_trials, int64_t sweeps_per_trial, int32_t exchange_every,
                     int32_t inserts_per_trial, double *temps_out, int32_t temps_cap, int32_t *R_out,
                     double *rates_out) {
  if (!ctx) return RFIM_EINVAL;
  rfim_ctx *c = ctx;
  if (n_trials < 0 || inserts_per_trial < 0 || exchange_every <= 0 || sweeps_per_trial < 0)
    return fail(c, RFIM_EINVAL, "invalid adaptation arguments");
  const int64_t R_final = (int64_t)c->R + (int64_t)n_trials * inserts_per_trial;
  if (R_final > c->Rcap) return fail(c, RFIM_EINVAL, "R_final %lld exceeds R_capacity %d", (long long)R_final, c->Rcap);
  if (temps_out && temps_cap < R_final) return fail(c, RFIM_EINVAL, "temps_cap %d < R_final %lld", temps_cap, (long long)R_final);
  if (c->plan.counter && !bits_plan_fits(c->plan, (int32_t)R_final))
    return fail(c, RFIM_EINVAL, "R_final %lld not supported by the bit-layout plan", (long long)R_final);
  int rc;
  for (int32_t t = 1; t <= n_trials; ++t) {
    if (inserts_per_trial > c->R - 1) return fail(c, RFIM_EINVAL, "more insertions than intervals");
    if ((rc = upload_temps(c))) return rc;
    if ((rc = reset_state(c, (uint32_t)t))) return rc;
    if ((rc = do_run(c, sweeps_per_trial, exchange_every, INT64_MAX))) return rc;
    const int32_t np = c->R - 1;
    std::vector<uint64_t> att(np), acc(np);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(att.data(), c->att, np * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(acc.data(), c->acc, np * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    std::vector<double> rate(np);
    for (int32_t k = 0; k < np; ++k) rate[k] = att[k] ? (double)acc[k] / (double)att[k] : 0.0;
    if (rates_out)
      for (int32_t k = 0; k < np; ++k) rates_out[(int64_t)(t - 1) * c->Rcap + k] = rate[k];
    // Sec. 4: exchange rates into a min-heap, the a lowest intervals get their midpoint.
    using Item = std::pair<double, int32_t>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int32_t k = 0; k < np; ++k) heap.push({rate[k], k});
    std::vector<double> added;
    for (int32_t a = 0; a < inserts_per_trial && !heap.empty(); ++a) {
      const int32_t k = heap.top().second;
      heap.pop();
      added.push_back(0.5 * (c->T[k] + c->T[k + 1]));
    }
    c->T.insert(c->T.end(), added.begin(), added.end());
    std::sort(c->T.begin(), c->T.end());
    c->R = (int32_t)c->T.size();
  }
  if ((rc = upload_temps(c))) return rc;
  if ((rc = reset_state(c, 0))) return rc;
  if (temps_out) std::copy(c->T.begin(), c->T.end(), temps_out);
  if (R_out) *R_out = c->R;
  return RFIM_OK;
}

int rfim_observables(rfim_ctx *ctx, rfim_obs *out) {
  if (!ctx || !out) return RFIM_EINVAL;
  rfim_ctx *c = ctx;
  if (int rc = check_device_error(c)) return rc;
  const int32_t R = c->R;
  std::vector<double> obs((size_t)R * 5);
  std::vector<uint64_t> att(R), acc(R);
  int64_t nm = 0;
  CUDA_OR_FAIL(c, cudaMemcpyAsync(obs.data(), c->obs, obs.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OR_FAIL(c, cudaMemcpyAsync(att.data(), c->att, R * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OR_FAIL(c, cudaMemcpyAsync(acc.data(), c->acc, R * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OR_FAIL(c, cudaMemcpyAsync(&nm, c->n_meas, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  out->R = R;
  out->n_meas = nm;
  double *cols[5] = {out->e, out->e2, out->absm, out->m2, out->m4};
  for (int q = 0; q < 5; ++q)
    if (cols[q])
      for (int32_t k = 0; k < R; ++k) cols[q][k] = obs[(size_t)k * 5 + q];
  if (out->T) std::copy(c->T.begin(), c->T.end(), out->T);
  if (out->att) std::copy(att.begin(), att.begin() + (R - 1), out->att);
  if (out->acc) std::copy(acc.begin(), acc.begin() + (R - 1), out->acc);
  if (out->F) {
    if (c->sumF) {
      CUDA_OR_FAIL(c, cudaMemcpyAsync(out->F, c->sumF, (size_t)R * 8, cudaMemcpyDeviceToHost, c->stream));
      CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    } else {
      std::fill(out->F, out->F + R, 0.0);
    }
  }
  return RFIM_OK;
}

int rfim_set_measure_xi(rfim_ctx *ctx, int32_t on) {
  if (!ctx) return RFIM_EINVAL;
  rfim_ctx *c = ctx;
  if (!on) {
    c->xi_on = false;
    return RFIM_OK;
  }
  int64_t nm = 0;
  CUDA_OR_FAIL(c, cudaMemcpyAsync(&nm, c->n_meas, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  if (nm > 0 && !c->xi_on) return fail(c, RFIM_ESTATE, "enable the structure-factor measurement before the first measurement");
  if (!c->sumF) {
    int rc;
    if ((rc = dalloc(c, &c->sumF, (size_t)c->Rcap))) return rc;
    if ((rc = dalloc(c, &c->kcos, (size_t)c->L))) return rc;
    if ((rc = dalloc(c, &c->ksin, (size_t)c->L))) return rc;
    std::vector<double> kc(c->L), ks(c->L);
    wave_tables(c->L, kc.data(), ks.data());
    CUDA_OR_FAIL(c, cudaMemcpy(c->kcos, kc.data(), c->L * 8, cudaMemcpyHostToDevice));
    CUDA_OR_FAIL(c, cudaMemcpy(c->ksin, ks.data(), c->L * 8, cudaMemcpyHostToDevice));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->sumF, 0, (size_t)c->Rcap * 8, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  }
  c->xi_on = true;
  return RFIM_OK;
}

int rfim_set_multihit(rfim_ctx *ctx, int32_t mh, int32_t tile) {
  if (!ctx) return RFIM_EINVAL;
  rfim_ctx *c = ctx;
  if (mh < 0) return fail(c, RFIM_EINVAL, "mh must be >= 0");
  if (mh == 0) {
    c->mh = MultiHit{};
    return RFIM_OK;
  }
  if (c->layout != RFIM_LAYOUT_BITPACK) return fail(c, RFIM_EINVAL, "multi-hit sweeps need the bit layout");
  if (!multihit_tile_ok(c->L, tile))
    return fail(c, RFIM_EINVAL, "tile must be 8, 16 or 32 with L in {16, 32, 64} divisible by 2 tile (L=%d, tile=%d)",
                c->L, tile);
  const bool bim = c->kind == kBimodal;
  if (prepare_multihit(c->plan, bim) != cudaSuccess) {
    cudaGetLastError();
    // the current launch shape has no multi-hit instance (e.g. the grid-wide plan): switch to the
    // default cluster / single-CTA shape of this L
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    const char *shape = c->L == 64 ? "4,4,4,512" : c->L == 32 ? "2,1,1,256" : "1,8,1,512";
    BitsPlan np;
    set_plan_override(shape);
    const int rc = make_bits_plan(c->L, c->Rcap, bim, &np, &c->err);
    set_plan_override(nullptr);
    if (rc) return rc;
    if (np.field4) {
      const cudaError_t e = build_field4(view_of(c), np, c->stream);
      if (e != cudaSuccess) {
        free_bits_plan(np);
        return fail(c, RFIM_ECUDA, "field4 kernel: %s", cudaGetErrorString(e));
      }
      c->launches += 1;
    }
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    free_bits_plan(c->plan);
    c->plan = np;
    CUDA_OR_FAIL(c, prepare_multihit(c->plan, bim));
  }
  c->mh = make_multihit(c->L, mh, tile);
  return RFIM_OK;
}

int rfim_thermal(const rfim_obs *obs, int32_t N, double *out) {
  if (!obs || !out || N < 1 || obs->R < 1 || !obs->T || !obs->e || !obs->e2 || !obs->absm || !obs->m2 || !obs->m4)
    return RFIM_EINVAL;
  const double nan = std::nan(""), n = (double)obs->n_meas;
  for (int32_t k = 0; k < obs->R; ++k) {
    double *o = out + (size_t)k * 7;
    if (obs->n_meas <= 0) {
      for (int q = 0; q < 7; ++q) o[q] = nan;
      continue;
    }
    const double e = obs->e[k] / n, e2 = obs->e2[k] / n, T = obs->T[k];
    o[0] = e;
    o[1] = (double)N / (T * T) * (e2 - e * e);
    o[2] = obs->absm[k] / n;
    o[3] = obs->m2[k] / n;
    o[4] = obs->m4[k] / n;
    if (obs->F) {
      // <F> below 1e-20 is the rounding of an exactly uniform lattice (a lattice with a spin
      // against the others has F >= 4/N per measurement): xi diverges
      const double F = obs->F[k] / n, arg = (double)N * o[3] / F - 1.0;
      o[5] = F;
      o[6] = F < 1e-20 ? HUGE_VAL : (arg >= 0.0 ? std::sqrt(arg) : nan);
    } else {
      o[5] = o[6] = nan;
    }
  }
  return RFIM_OK;
}

int rfim_disorder_average(const double *thermals, int32_t n, int32_t R, double *out) {
  if (!thermals || !out || n < 1 || R < 1) return RFIM_EINVAL;
  for (int32_t k = 0; k < R; ++k) {
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int32_t i = 0; i < n; ++i)
      for (int q = 0; q < 7; ++q) s[q] += thermals[((size_t)i * R + k) * 7 + q];
    for (int q = 0; q < 7; ++q) s[q] /= (double)n;
    double *o = out + (size_t)k * 5;
    o[0] = s[0];
    o[1] = s[1];
    o[2] = s[2];
    o[3] = s[6];
    o[4] = 0.5 * (3.0 - s[4] / (s[3] * s[3]));
  }
  return RFIM_OK;
}

int rfim_get_state(rfim_ctx *ctx, int8_t *spins, int32_t *t2r, double *E, int64_t *sweep, int64_t *xstep) {
  if (!ctx) return RFIM_EINVAL;
  rfim_ctx *c = ctx;
  if (int rc = check_device_error(c)) return rc;
  const size_t RN = (size_t)c->R * c->N;
  RealView v = view_of(c);
  if (spins) {
    if (!c->scratch8) {
      int rc = dalloc(c, &c->scratch8, (size_t)c->Rcap * c->N);
      if (rc) return rc;
    }
    CUDA_OR_FAIL(c, launch_to_natural(v, c->R, c->layout == RFIM_LAYOUT_BITPACK, c->scratch8, c->stream));
    c->launches += 1;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(spins, c->scratch8, RN, cudaMemcpyDeviceToHost, c->stream));
  }
  if (t2r) CUDA_OR_FAIL(c, cudaMemcpyAsync(t2r, c->t2r, c->R * 4, cudaMemcpyDeviceToHost, c->stream));
  if (E) {
    // recompute from the current spins into the energy buffer, then read it
    CUDA_OR_FAIL(c, launch_energy(v, (double)c->J, (double)c->h, c->layout == RFIM_LAYOUT_BITPACK, c->stream,
                                 c->eparts.count ? &c->eparts : nullptr));
    c->launches += 1;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(E, c->E, c->R * 8, cudaMemcpyDeviceToHost, c->stream));
  }
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  if (sweep) *sweep = c->sweep;
  if (xstep) *xstep = c->xstep;
  return RFIM_OK;
}

int rfim_set_state(rfim_ctx *ctx, const int8_t *spins, const int32_t *t2r, int64_t sweep, int64_t xstep) {
  if (!ctx) return RFIM_EINVAL;
  rfim_ctx *c = ctx;
  if (sweep < 0 || xstep < 0) return fail(c, RFIM_EINVAL, "negative counter");
  const size_t RN = (size_t)c->R * c->N;
  if (spins)
    for (size_t i = 0; i < RN; ++i)
      if (spins[i] != 1 && spins[i] != -1) return fail(c, RFIM_EINVAL, "spin %zu is not +-1", i);
  std::vector<int32_t> r2t;
  if (t2r) {
    r2t.assign(c->R, -1);
    for (int32_t k = 0; k < c->R; ++k) {
      if (t2r[k] < 0 || t2r[k] >= c->R || r2t[t2r[k]] != -1) return fail(c, RFIM_EINVAL, "t2r is not a permutation");
      r2t[t2r[k]] = k;
    }
  }
  RealView v = view_of(c);
  if (spins) {
    if (!c->scratch8) {
      int rc = dalloc(c, &c->scratch8, (size_t)c->Rcap * c->N);
      if (rc) return rc;
    }
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->scratch8, spins, RN, cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, launch_from_natural(v, c->R, c->layout == RFIM_LAYOUT_BITPACK, c->scratch8, c->stream));
    c->launches += 1;
  }
  if (t2r) {
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->t2r, t2r, c->R * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->r2t, r2t.data(), c->R * 4, cudaMemcpyHostToDevice, c->stream));
  }
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  c->sweep = sweep;
  c->xstep = xstep;
  return RFIM_OK;
}

int rfim_get_field(rfim_ctx *ctx, float *h_out) {
  if (!ctx || !h_out) return RFIM_EINVAL;
  CUDA_OR_FAIL(ctx, cudaMemcpyAsync(h_out, ctx->hraw, (size_t)ctx->N * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  return RFIM_OK;
}

const char *rfim_last_error(const rfim_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int64_t rfim_launch_count(const rfim_ctx *ctx) { return ctx ? ctx->launches : 0; }

int rfim_get_plan(const rfim_ctx *ctx, char *plan_out, int32_t plan_cap) {
  if (!ctx || !plan_out || plan_cap < 1) return RFIM_EINVAL;
  const BitsPlan &p = ctx->plan;
  if (!p.counter) {
    plan_out[0] = '\0';
    return RFIM_OK;
  }
  snprintf(plan_out, (size_t)plan_cap, "%d,%d,%d,%d%s%s", p.S, p.G, p.GT, p.threads, p.NS == 4 ? ",4" : "",
           p.i8 ? ",int8" : "");
  return RFIM_OK;
}

int rfim_tune(int32_t L, int32_t R, int32_t field_kind, char *plan_out, int32_t plan_cap, double *attempts_per_ns) {
  if (!bits_supported(L) || R < 2 || field_kind < 0 || field_kind > 2)
    return fail(nullptr, RFIM_EINVAL, "rfim_tune: L in {8,16,32,64}, R >= 2, known field kind");
  const bool bim = field_kind == RFIM_FIELD_BIMODAL;
  std::vector<double> T(R);
  for (int32_t k = 0; k < R; ++k) T[k] = 1.0 * std::pow(5.0, (double)k / (R - 1));
  std::vector<float> field;
  if (field_kind == RFIM_FIELD_EXPLICIT) field.assign((size_t)L * L * L, 0.5f);
  rfim_config cfg{};
  cfg.L = L;
  cfg.R = R;
  cfg.R_capacity = R;
  cfg.J = 1.0f;
  cfg.h = 1.0f;
  cfg.field_kind = field_kind;
  cfg.field = field.empty() ? nullptr : field.data();
  cfg.field_seed = 1;
  cfg.seed = 7;
  cfg.temps = T.data();
  cfg.layout = RFIM_LAYOUT_BITPACK;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return fail(nullptr, RFIM_ECUDA, "rfim_tune: stream");
  cfg.stream = st;
  const int64_t intervals = L >= 32 ? 20 : 50, ex = 10;
  std::string best;
  double best_rate = 0.0;
  for (const std::string &cand : plan_candidates(L)) {
    set_plan_override(cand.c_str());
    rfim_ctx *c = nullptr;
    const int rc = rfim_create(&cfg, &c);
    set_plan_override(nullptr);
    if (rc != RFIM_OK) continue;  // shape not available for this R (or does not fit)
    double ms = 0.0;
    int64_t launches = 0;
    bool ok = do_run(c, 2 * ex, ex, INT64_MAX) == RFIM_OK && rfim_profile(c, 1) == RFIM_OK &&
              do_run(c, intervals * ex, ex, INT64_MAX) == RFIM_OK &&
              rfim_profile_read(c, &ms, &launches, nullptr, nullptr) == RFIM_OK && ms > 0.0;
    rfim_destroy(c);
    if (!ok) continue;
    const double rate = (double)L * L * L * R * intervals * ex / (ms * 1e6);
    if (rate > best_rate) {
      best_rate = rate;
      best = cand;
    }
  }
  cudaStreamDestroy(st);
  if (best.empty()) return fail(nullptr, RFIM_ECUDA, "rfim_tune: no launch shape ran");
  remember_tuned_plan(L, R, bim, best);
  if (plan_out && plan_cap > 0) snprintf(plan_out, plan_cap, "%s", best.c_str());
  if (attempts_per_ns) *attempts_per_ns = best_rate;
  return RFIM_OK;
}

int rfim_profile(rfim_ctx *ctx, int enable) {
  if (!ctx) return RFIM_EINVAL;
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto &v : ctx->ev_used) {
    for (auto &p : v) ctx->ev_free.push_back(p);
    v.clear();
  }
  ctx->prof_units[0] = ctx->prof_units[1] = 0;
  ctx->profiling = enable != 0;
  return RFIM_OK;
}

int rfim_profile_read(rfim_ctx *ctx, double *sweep_ms, int64_t *sweep_launches, double *exchange_ms,
                      int64_t *exchange_launches) {
  if (!ctx) return RFIM_EINVAL;
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  double tot[2] = {0.0, 0.0};
  for (int k = 0; k < 2; ++k)
    for (auto &p : ctx->ev_used[k]) {
      float ms = 0.f;
      CUDA_OR_FAIL(ctx, cudaEventElapsedTime(&ms, p.first, p.second));
      tot[k] += ms;
    }
  if (sweep_ms) *sweep_ms = tot[0];
  if (sweep_launches) *sweep_launches = ctx->prof_units[0];
  if (exchange_ms) *exchange_ms = tot[1];
  if (exchange_launches) *exchange_launches = ctx->prof_units[1];
  return RFIM_OK;
}

}  // extern "C"
