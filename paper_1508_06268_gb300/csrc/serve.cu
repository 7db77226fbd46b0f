// Serving runtime: continuous batching of independent disorder realizations (the quenched
// average of Sec. 7 needs many of them).  Requests are admitted as slots and device memory free
// up; every resident realization advances by a fixed number of exchange intervals per launch of a
// captured CUDA graph of persistent batched kernels (kernels_batch.cu); finished realizations are
// retired between graph launches and their observables kept until polled.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "rfim.h"
#include "batch.h"
#include "internal.h"
#include "sweep_bits.h"

using namespace rfim;

namespace {

using Clock = std::chrono::steady_clock;

double seconds(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

// First-fit sub-allocator over one device allocation (256-byte granules, coalescing frees), so
// admitting and retiring realizations never calls cudaMalloc / cudaFree (which synchronise).
struct Arena {
  char *base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }
  size_t alloc(size_t bytes) {
    bytes = round(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    bytes = round(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

constexpr int kMaxServedR = 1024;
constexpr int kMaxItemsPerSlot = 512;  // kMaxServedR / smallest replica group (2)

struct Request {
  uint64_t ticket = 0;
  rfim_config cfg{};
  std::vector<double> temps;
  std::vector<float> field;
  int64_t sweeps = 0;
  int32_t ex = 0;
  int64_t measure_from = 0;
  Clock::time_point arrival;
};

struct Result {
  int code = RFIM_OK;
  std::string msg;
  int32_t R = 0;
  std::vector<double> T, obs, F;
  std::vector<uint64_t> att, acc;
  int64_t n_meas = 0;
  double latency_s = 0.0, queued_s = 0.0;
};

struct Slot {
  bool used = false;
  uint64_t ticket = 0;
  int32_t L = 0, R = 0, N = 0;
  size_t off = 0, bytes = 0;
  SlotDesc desc{};
  Clock::time_point arrival, admitted;
  std::vector<double> T;
  int64_t attempts = 0;
};

// Replicas per work item and per thread for each L in batched launches (S = 1: whole replicas).
struct BatchShape {
  int G, GT;
};
using ShapeMap = std::map<int, BatchShape>;

// Built-in shapes, used until rfim_server_tune has measured better ones in this process.
ShapeMap default_shapes() { return {{64, {2, 2}}, {32, {8, 2}}, {16, {16, 1}}, {8, {16, 1}}}; }

bool shape_ok(int L, int G, int GT) {
  return batch_supported(L, GT) && G >= GT && G % GT == 0 && G <= 1024 && batch_smem(L, G) <= (size_t)227 * 1024;
}

// "L:G:GT,..." over the defaults; false if an entry is malformed or names no batched instance.
bool parse_shapes(const char *text, ShapeMap *out) {
  ShapeMap m = default_shapes();
  if (text && *text) {
    const std::string str(text);
    size_t pos = 0;
    for (;;) {
      int l = 0, g = 0, gt = 0, used = 0;
      if (sscanf(str.c_str() + pos, "%d:%d:%d%n", &l, &g, &gt, &used) != 3 || !shape_ok(l, g, gt)) return false;
      m[l] = {g, gt};
      pos += (size_t)used;
      if (pos >= str.size()) break;
      if (str[pos] != ',') return false;
      ++pos;
    }
  }
  *out = m;
  return true;
}

std::string format_shapes(const ShapeMap &m) {
  std::string r;
  for (auto it = m.rbegin(); it != m.rend(); ++it) {
    if (!r.empty()) r += ",";
    r += std::to_string(it->first) + ":" + std::to_string(it->second.G) + ":" + std::to_string(it->second.GT);
  }
  return r;
}

// Result of the last rfim_server_tune in this process (empty: none).
std::mutex g_tuned_mu;
std::string g_tuned_shapes;
int g_tuned_intervals = 0;

}  // namespace

struct rfim_server {
  int device = 0;
  cudaStream_t stream = nullptr;
  Arena arena;
  int max_slots = 0, K = 1, grid = 0;
  size_t smem = 0;
  SlotDesc *d_slots = nullptr;
  SlotCtl *d_ctls = nullptr;
  BatchItem *d_items = nullptr;
  BatchQueue *d_queue = nullptr;
  unsigned int *d_err = nullptr;  // device error word of the batched launches (debug-build checks)
  std::vector<Slot> slots;
  std::vector<SlotCtl> h_ctls;
  std::deque<Request> pending;
  std::map<uint64_t, Result> done;
  uint64_t next_ticket = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::string err;
  int fatal = RFIM_OK;
  int64_t graph_launches = 0, completed = 0, resident = 0;
  double busy_s = 0.0, attempts = 0.0;
  bool items_dirty = true;
  bool measure_xi = false;
  ShapeMap shapes;  // (G, GT) per L of this server's batched launches
};

namespace {

thread_local std::string g_server_error;

// Copies on the server's own stream (never the legacy default stream), then waits for them.
cudaError_t copy_sync(rfim_server *s, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, s->stream);
  return e == cudaSuccess ? cudaStreamSynchronize(s->stream) : e;
}

int server_fail(rfim_server *s, int code, const std::string &msg) {
  if (s)
    s->err = msg;
  else
    g_server_error = msg;
  return code;
}

size_t slot_bytes(int32_t L, int32_t R, int32_t kind, bool xi) {
  const size_t N = (size_t)L * L * L, W = N / 64, wpad = (W + 31) / 32 * 32;
  size_t b = 0;
  auto add = [&](size_t x) { b += Arena::round(x); };
  add((size_t)R * 2 * W * 4);                         // bits
  add(2 * W * 4);                                     // hbits
  if (kind != kBimodal) { add(2 * wpad * 8 * 16); add(2 * 10 * wpad * 16); add(sizeof(FieldQuant)); }  // field4, limbs
  add(N * 4); add(N * 4); add(N);                     // hraw, hh_c, hbit_c
  add((size_t)R * 32 * 4); add(32); add(R * 4); add(R * 4); add(R * 8);  // thr gjn b2 b2l beta
  add(R * 4); add(R * 4); add(R * 8); add(R * 8); add(R * 8); add(R * 8);  // t2r r2t E M att acc
  add((size_t)R * 40); add(8);                        // obs n_meas
  add(R * 8); add(R * 8); add(R * 8); add(R * 8); add(4);  // partials, counter
  if (xi) { add(R * 8); add(R * 8); add(L * 8); add(L * 8); }  // Fr sumF kcos ksin
  return b;
}

// Builds a resident realization in arena memory and fills its descriptor (stream idle).
int init_slot(rfim_server *s, Slot &sl, const Request &rq) {
  const rfim_config &c = rq.cfg;
  const int32_t L = c.L, R = c.R;
  const size_t N = (size_t)L * L * L, W = N / 64, wpad = (W + 31) / 32 * 32;
  char *p = s->arena.base + sl.off;
  auto take = [&](size_t bytes) {
    char *q = p;
    p += Arena::round(bytes);
    return (void *)q;
  };
  RealView v{};
  v.L = L; v.Lh = L / 2; v.N = (int32_t)N; v.R = R; v.kind = c.field_kind;
  v.seed = c.seed; v.realization = c.realization; v.stage = 0;
  v.bits = (uint32_t *)take((size_t)R * 2 * W * 4);
  uint32_t *hbits = (uint32_t *)take(2 * W * 4);
  float4 *field4 = c.field_kind != kBimodal ? (float4 *)take(2 * wpad * 8 * 16) : nullptr;
  uint4 *flimb = field4 ? (uint4 *)take(2 * 10 * wpad * 16) : nullptr;
  FieldQuant *fquant = field4 ? (FieldQuant *)take(sizeof(FieldQuant)) : nullptr;
  float *hraw = (float *)take(N * 4);
  float *hh_c = (float *)take(N * 4);
  uint8_t *hbit_c = (uint8_t *)take(N);
  uint32_t *thr = (uint32_t *)take((size_t)R * 32 * 4);
  float *gjn = (float *)take(32);
  float *b2 = (float *)take(R * 4);
  float *b2l = (float *)take(R * 4);
  double *beta = (double *)take(R * 8);
  v.t2r = (int32_t *)take(R * 4);
  v.r2t = (int32_t *)take(R * 4);
  v.E = (double *)take(R * 8);
  v.M = (int64_t *)take(R * 8);
  v.att = (uint64_t *)take(R * 8);
  v.acc = (uint64_t *)take(R * 8);
  v.obs = (double *)take((size_t)R * 40);
  v.n_meas = (int64_t *)take(8);
  ExchArgs xa{};
  xa.partB = (long long *)take(R * 8);
  xa.partM = (long long *)take(R * 8);
  xa.partFi = (long long *)take(R * 8);
  xa.partF = (double *)take(R * 8);
  xa.counter = (unsigned int *)take(4);
  xa.err = s->d_err;
  double *kwave = nullptr;
  if (s->measure_xi) {
    xa.Fr = (double *)take(R * 8);
    xa.sumF = (double *)take(R * 8);
    kwave = (double *)take(L * 8);
    double *ks = (double *)take(L * 8);
    xa.kcos = kwave;
    xa.ksin = ks;
  }
  v.hh_c = hh_c; v.hbit_c = hbit_c; v.hbits = hbits; v.thr = thr; v.gjn = gjn; v.b2 = b2; v.b2l = b2l;
  v.beta_d = beta;

  cudaStream_t st = s->stream;
  auto ck = [&](cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
      s->err = std::string(what) + ": " + cudaGetErrorString(e);
      return false;
    }
    return true;
  };
  if (c.field_kind == RFIM_FIELD_EXPLICIT &&
      !ck(cudaMemcpyAsync(hraw, rq.field.data(), N * 4, cudaMemcpyHostToDevice, st), "field upload"))
    return RFIM_ECUDA;
  if (!ck(launch_field(v, c.field_kind, c.field_seed, c.h, hraw, hh_c, hbit_c, hbits, st), "field")) return RFIM_ECUDA;
  if (field4) {
    BitsPlan tmp;
    tmp.field4 = field4;
    tmp.flimb = flimb;
    tmp.fquant = fquant;
    const cudaError_t e = build_field4(v, tmp, st);
    tmp.field4 = nullptr;  // owned by the arena
    tmp.flimb = nullptr;
    tmp.fquant = nullptr;
    if (!ck(e, "field4")) return RFIM_ECUDA;
    xa.flimb = flimb;
    xa.fquant = fquant;
  }
  if (!ck(launch_init_spins(v, R, 0, true, st), "init")) return RFIM_ECUDA;
  std::vector<uint32_t> thr_h((size_t)R * 32);
  std::vector<float> b2_h(R), b2l_h(R);
  std::vector<double> beta_h(R);
  float gjn_h[8];
  temperature_tables(rq.temps.data(), R, c.J, c.h, thr_h.data(), b2_h.data(), b2l_h.data(), beta_h.data(), gjn_h);
  std::vector<int32_t> id(R);
  std::iota(id.begin(), id.end(), 0);
  std::vector<double> wave(2 * (size_t)L);
  if (kwave) wave_tables(L, wave.data(), wave.data() + L);
  bool ok = ck(cudaMemcpyAsync(thr, thr_h.data(), thr_h.size() * 4, cudaMemcpyHostToDevice, st), "tables") &&
            ck(cudaMemcpyAsync(b2, b2_h.data(), R * 4, cudaMemcpyHostToDevice, st), "tables") &&
            ck(cudaMemcpyAsync(b2l, b2l_h.data(), R * 4, cudaMemcpyHostToDevice, st), "tables") &&
            ck(cudaMemcpyAsync(beta, beta_h.data(), R * 8, cudaMemcpyHostToDevice, st), "tables") &&
            ck(cudaMemcpyAsync(gjn, gjn_h, 32, cudaMemcpyHostToDevice, st), "tables") &&
            ck(cudaMemcpyAsync(v.t2r, id.data(), R * 4, cudaMemcpyHostToDevice, st), "perm") &&
            ck(cudaMemcpyAsync(v.r2t, id.data(), R * 4, cudaMemcpyHostToDevice, st), "perm") &&
            ck(cudaMemsetAsync(v.E, 0, R * 8, st), "zero") && ck(cudaMemsetAsync(v.M, 0, R * 8, st), "zero") &&
            ck(cudaMemsetAsync(v.att, 0, R * 8, st), "zero") && ck(cudaMemsetAsync(v.acc, 0, R * 8, st), "zero") &&
            ck(cudaMemsetAsync(v.obs, 0, (size_t)R * 40, st), "zero") &&
            ck(cudaMemsetAsync(v.n_meas, 0, 8, st), "zero") && ck(cudaMemsetAsync(xa.counter, 0, 4, st), "zero") &&
            (!kwave || (ck(cudaMemsetAsync(xa.sumF, 0, R * 8, st), "zero") &&
                        ck(cudaMemcpyAsync(kwave, wave.data(), L * 8, cudaMemcpyHostToDevice, st), "tables") &&
                        ck(cudaMemcpyAsync((void *)xa.ksin, wave.data() + L, L * 8, cudaMemcpyHostToDevice, st), "tables"))) &&
            ck(cudaStreamSynchronize(st), "slot init");
  if (!ok) return RFIM_ECUDA;
  const BatchShape sh = s->shapes.at(L);
  xa.J = (double)c.J;
  xa.h = (double)c.h;
  sl.desc = SlotDesc{};
  sl.desc.v = v;
  sl.desc.field4 = field4;
  sl.desc.xa = xa;
  sl.desc.L = L;
  sl.desc.kind = c.field_kind == kBimodal ? kBimodal : kGaussian;
  sl.desc.G = std::min(sh.G, R);
  sl.desc.GT = sh.GT;
  if (sl.desc.G % sl.desc.GT) sl.desc.GT = 1;
  sl.desc.nitems = (R + sl.desc.G - 1) / sl.desc.G;
  return RFIM_OK;
}

// Retires finished realizations (reads their observables), admits pending requests while slots
// and arena memory allow, and refreshes the device descriptors and work queue.  Stream idle.
void refresh(rfim_server *s) {
  for (int i = 0; i < s->max_slots; ++i) {
    Slot &sl = s->slots[i];
    if (!sl.used || s->h_ctls[i].intervals_left > 0) continue;
    Result res;
    const RealView &v = sl.desc.v;
    res.R = sl.R;
    res.T = sl.T;
    res.obs.resize((size_t)sl.R * 5);
    res.att.resize(sl.R);
    res.acc.resize(sl.R);
    copy_sync(s, res.obs.data(), v.obs, res.obs.size() * 8, cudaMemcpyDeviceToHost);
    copy_sync(s, res.att.data(), v.att, sl.R * 8, cudaMemcpyDeviceToHost);
    copy_sync(s, res.acc.data(), v.acc, sl.R * 8, cudaMemcpyDeviceToHost);
    copy_sync(s, &res.n_meas, v.n_meas, 8, cudaMemcpyDeviceToHost);
    if (sl.desc.xa.sumF) {
      res.F.resize(sl.R);
      copy_sync(s, res.F.data(), sl.desc.xa.sumF, sl.R * 8, cudaMemcpyDeviceToHost);
    }
    const Clock::time_point now = Clock::now();
    res.latency_s = seconds(sl.arrival, now);
    res.queued_s = seconds(sl.arrival, sl.admitted);
    s->attempts += (double)sl.attempts;
    s->arena.release(sl.off, sl.bytes);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      sl.used = false;
      s->completed += 1;
      s->resident -= 1;
      s->done[sl.ticket] = std::move(res);
    }
    s->items_dirty = true;
  }
  for (;;) {
    Request rq;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->pending.empty()) break;
      int free_slot = -1;
      for (int i = 0; i < s->max_slots; ++i)
        if (!s->slots[i].used) {
          free_slot = i;
          break;
        }
      if (free_slot < 0) break;
      const Request &front = s->pending.front();
      const size_t need = slot_bytes(front.cfg.L, front.cfg.R, front.cfg.field_kind, s->measure_xi);
      if (need > s->arena.size) {
        Result bad;
        bad.code = RFIM_ENOMEM;
        bad.msg = "realization larger than the server's memory budget";
        s->done[front.ticket] = bad;
        s->pending.pop_front();
        continue;
      }
      const size_t off = s->arena.alloc(need);
      if (off == SIZE_MAX) break;  // wait for retirements
      rq = std::move(s->pending.front());
      s->pending.pop_front();
      Slot &sl = s->slots[free_slot];
      sl.used = true;
      s->resident += 1;
      sl.ticket = rq.ticket;
      sl.L = rq.cfg.L;
      sl.R = rq.cfg.R;
      sl.N = rq.cfg.L * rq.cfg.L * rq.cfg.L;
      sl.off = off;
      sl.bytes = need;
      sl.arrival = rq.arrival;
      sl.admitted = Clock::now();
      sl.T = rq.temps;
      sl.attempts = (int64_t)sl.N * sl.R * rq.sweeps;
      rq.cfg.temps = nullptr;
      rq.cfg.field = nullptr;
      const int rc = init_slot(s, sl, rq);
      if (rc != RFIM_OK) {
        Result bad;
        bad.code = rc;
        bad.msg = s->err;
        s->done[rq.ticket] = bad;
        s->arena.release(off, need);
        sl.used = false;
        s->resident -= 1;
        continue;
      }
      SlotCtl ctl{};
      ctl.sweep0 = 0;
      ctl.j = 0;
      ctl.intervals_left = (int32_t)(rq.sweeps / rq.ex);
      ctl.nsw = rq.ex;
      ctl.measure_from = rq.measure_from;
      s->h_ctls[free_slot] = ctl;
      copy_sync(s, s->d_ctls + free_slot, &ctl, sizeof ctl, cudaMemcpyHostToDevice);
      s->items_dirty = true;
    }
  }
  if (!s->items_dirty) return;
  std::vector<BatchItem> items;
  for (int i = 0; i < s->max_slots; ++i) {
    Slot &sl = s->slots[i];
    if (!sl.used) continue;
    for (int r0 = 0; r0 < sl.R; r0 += sl.desc.G) items.push_back(BatchItem{i, r0, std::min(sl.desc.G, sl.R - r0), 0});
    copy_sync(s, s->d_slots + i, &sl.desc, sizeof(SlotDesc), cudaMemcpyHostToDevice);
  }
  // largest items first so that the long ones start early
  std::stable_sort(items.begin(), items.end(), [&](const BatchItem &a, const BatchItem &b) {
    return (int64_t)a.gact * s->slots[a.slot].N > (int64_t)b.gact * s->slots[b.slot].N;
  });
  if (!items.empty()) copy_sync(s, s->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
  BatchQueue q{0u, 0u, (int32_t)items.size(), 0};
  copy_sync(s, s->d_queue, &q, sizeof q, cudaMemcpyHostToDevice);
  s->items_dirty = false;
}

void worker_loop(rfim_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) return;
    }
    refresh(s);
    bool active = false;
    for (int i = 0; i < s->max_slots; ++i) active |= s->slots[i].used && s->h_ctls[i].intervals_left > 0;
    if (!active) {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) return;
      s->cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return s->stop || !s->pending.empty(); });
      continue;
    }
    const Clock::time_point t0 = Clock::now();
    cudaError_t e = cudaGraphLaunch(s->gexec, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess)
      e = copy_sync(s, s->h_ctls.data(), s->d_ctls, sizeof(SlotCtl) * s->max_slots, cudaMemcpyDeviceToHost);
    if (kDebugBuild && e == cudaSuccess) {  // debug build: bounds checks of this replay
      unsigned int word = 0;
      e = copy_sync(s, &word, s->d_err, 4, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && word) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->fatal = RFIM_EBOUNDS;
        s->err = "batched launch: a bounds check of the debug build failed";
        return;
      }
    }
    s->busy_s += seconds(t0, Clock::now());
    s->graph_launches += 1;
    if (e != cudaSuccess) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->fatal = RFIM_ECUDA;
      s->err = std::string("batched launch: ") + cudaGetErrorString(e);
      return;
    }
  }
}

void destroy_server(rfim_server *s) {
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv.notify_all();
    s->worker.join();
  }
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->graph) cudaGraphDestroy(s->graph);
  void *ptrs[] = {s->arena.base, s->d_slots, s->d_ctls, s->d_items, s->d_queue, s->d_err};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // namespace

extern "C" {

int rfim_server_create(const rfim_server_config *cfg, rfim_server **out) {
  if (!cfg || !out) return server_fail(nullptr, RFIM_EINVAL, "null argument");
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->intervals_per_launch < 0 || cfg->mem_budget_bytes < (1u << 20))
    return server_fail(nullptr, RFIM_EINVAL, "invalid server configuration");
  std::string tuned_shapes;
  int tuned_k = 0;
  {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    tuned_shapes = g_tuned_shapes;
    tuned_k = g_tuned_intervals;
  }
  ShapeMap shapes;
  if (!parse_shapes(cfg->batch_shapes ? cfg->batch_shapes : tuned_shapes.c_str(), &shapes))
    return server_fail(nullptr, RFIM_EINVAL, "batch_shapes: expected \"L:G:GT,...\" naming batched instances");
  rfim_server *s = new rfim_server();
  cudaGetDevice(&s->device);
  s->shapes = shapes;
  s->max_slots = cfg->max_slots;
  s->K = cfg->intervals_per_launch > 0 ? cfg->intervals_per_launch : (tuned_k > 0 ? tuned_k : 4);
  s->measure_xi = cfg->measure_xi != 0;
  s->slots.resize(s->max_slots);
  s->h_ctls.assign(s->max_slots, SlotCtl{});
  auto bail = [&](int code, const std::string &msg) {
    g_server_error = msg;
    cudaGetLastError();
    destroy_server(s);
    return code;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(RFIM_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
  e = cudaMalloc(&s->arena.base, cfg->mem_budget_bytes);
  if (e != cudaSuccess) return bail(RFIM_ENOMEM, std::string("arena: ") + cudaGetErrorString(e));
  s->arena.size = cfg->mem_budget_bytes;
  s->arena.free_[0] = cfg->mem_budget_bytes;
  const size_t nitems_max = (size_t)s->max_slots * kMaxItemsPerSlot;
  if ((e = cudaMalloc(&s->d_slots, sizeof(SlotDesc) * s->max_slots)) != cudaSuccess ||
      (e = cudaMalloc(&s->d_ctls, sizeof(SlotCtl) * s->max_slots)) != cudaSuccess ||
      (e = cudaMalloc(&s->d_items, sizeof(BatchItem) * nitems_max)) != cudaSuccess ||
      (e = cudaMalloc(&s->d_queue, sizeof(BatchQueue))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_err, sizeof(unsigned int))) != cudaSuccess)
    return bail(RFIM_ENOMEM, std::string("tables: ") + cudaGetErrorString(e));
  cudaMemsetAsync(s->d_err, 0, sizeof(unsigned int), s->stream);
  cudaMemsetAsync(s->d_ctls, 0, sizeof(SlotCtl) * s->max_slots, s->stream);
  cudaMemsetAsync(s->d_queue, 0, sizeof(BatchQueue), s->stream);
  cudaStreamSynchronize(s->stream);
  for (const auto &kv : s->shapes) s->smem = std::max(s->smem, batch_smem(kv.first, kv.second.G));
  if ((e = batch_prepare(s->smem)) != cudaSuccess) return bail(RFIM_ECUDA, std::string("attr: ") + cudaGetErrorString(e));
  int per_sm = 0, sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  if ((e = batch_occupancy(s->smem, &per_sm)) != cudaSuccess || per_sm < 1)
    return bail(RFIM_ECUDA, "batched kernel does not fit on an SM");
  s->grid = sms * per_sm;
  // capture K persistent launches once; every later step replays the graph
  e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
  for (int k = 0; k < s->K && e == cudaSuccess; ++k)
    e = launch_batch(s->grid, s->smem, s->d_slots, s->d_ctls, s->d_items, s->d_queue, s->stream);
  cudaError_t e2 = cudaStreamEndCapture(s->stream, &s->graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&s->gexec, s->graph, 0);
  if (e != cudaSuccess) return bail(RFIM_ECUDA, std::string("graph: ") + cudaGetErrorString(e));
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return RFIM_OK;
}

int rfim_server_submit(rfim_server *s, const rfim_config *cfg, int64_t n_sweeps, int32_t exchange_every,
                       int64_t measure_from, uint64_t *ticket) {
  if (!s || !cfg || !ticket) return server_fail(s, RFIM_EINVAL, "null argument");
  if (!bits_supported(cfg->L)) return server_fail(s, RFIM_EINVAL, "server supports L in {8,16,32,64}");
  if (cfg->R < 2 || cfg->R > kMaxServedR || !cfg->temps)
    return server_fail(s, RFIM_EINVAL, "R must be in [2, 1024] with a temperature set");
  if (cfg->field_kind < 0 || cfg->field_kind > 2 || (cfg->field_kind == RFIM_FIELD_EXPLICIT && !cfg->field))
    return server_fail(s, RFIM_EINVAL, "invalid field");
  if (exchange_every < 1 || n_sweeps < exchange_every || n_sweeps % exchange_every)
    return server_fail(s, RFIM_EINVAL, "n_sweeps must be a positive multiple of exchange_every");
  for (int32_t k = 0; k < cfg->R; ++k)
    if (!(cfg->temps[k] > 0.0) || (k && !(cfg->temps[k] > cfg->temps[k - 1])))
      return server_fail(s, RFIM_EINVAL, "temperatures must be positive and strictly ascending");
  Request rq;
  rq.cfg = *cfg;
  rq.temps.assign(cfg->temps, cfg->temps + cfg->R);
  if (cfg->field_kind == RFIM_FIELD_EXPLICIT) rq.field.assign(cfg->field, cfg->field + (size_t)cfg->L * cfg->L * cfg->L);
  rq.sweeps = n_sweeps;
  rq.ex = exchange_every;
  rq.measure_from = measure_from;
  rq.arrival = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal) return server_fail(s, s->fatal, s->err);
    rq.ticket = s->next_ticket++;
    *ticket = rq.ticket;
    s->pending.push_back(std::move(rq));
  }
  s->cv.notify_all();
  return RFIM_OK;
}

int rfim_server_poll(rfim_server *s, uint64_t ticket, rfim_obs *out, double *latency_s) {
  if (!s) return RFIM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    if (s->fatal) return server_fail(s, s->fatal, s->err);
    if (ticket == 0 || ticket >= s->next_ticket) return server_fail(s, RFIM_EINVAL, "unknown ticket");
    return RFIM_EBUSY;
  }
  const Result &r = it->second;
  if (r.code != RFIM_OK) {
    s->err = r.msg;
    const int code = r.code;
    s->done.erase(it);
    return code;
  }
  if (out) {
    out->R = r.R;
    out->n_meas = r.n_meas;
    double *cols[5] = {out->e, out->e2, out->absm, out->m2, out->m4};
    for (int q = 0; q < 5; ++q)
      if (cols[q])
        for (int32_t k = 0; k < r.R; ++k) cols[q][k] = r.obs[(size_t)k * 5 + q];
    if (out->T) std::copy(r.T.begin(), r.T.end(), out->T);
    if (out->att) std::copy(r.att.begin(), r.att.begin() + (r.R - 1), out->att);
    if (out->acc) std::copy(r.acc.begin(), r.acc.begin() + (r.R - 1), out->acc);
    if (out->F) {
      if (r.F.empty())
        std::fill(out->F, out->F + r.R, 0.0);
      else
        std::copy(r.F.begin(), r.F.end(), out->F);
    }
  }
  if (latency_s) *latency_s = r.latency_s;
  s->done.erase(it);
  return RFIM_OK;
}

int rfim_server_stats(rfim_server *s, rfim_server_info *out) {
  if (!s || !out) return RFIM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->queued = (int64_t)s->pending.size();
  out->resident = s->resident;
  out->completed = s->completed;
  out->graph_launches = s->graph_launches;
  out->busy_s = s->busy_s;
  out->attempts = s->attempts;
  out->grid = s->grid;
  out->intervals_per_launch = s->K;
  const std::string sh = format_shapes(s->shapes);
  snprintf(out->batch_shapes, sizeof out->batch_shapes, "%s", sh.c_str());
  return RFIM_OK;
}

int rfim_server_destroy(rfim_server *s) {
  if (!s) return RFIM_OK;
  destroy_server(s);
  return RFIM_OK;
}

const char *rfim_server_last_error(const rfim_server *s) { return s ? s->err.c_str() : g_server_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Tuner of the batched kernel: launch shape (replicas per work item G, per thread GT) for each L,
// then exchange intervals per graph replay, each timed closed-loop on scratch realizations.
namespace {

struct MixEntry {
  int L, R;
};

// Wall-clock attempts/ns of `stream` submitted at once to a fresh server (second of two passes).
int time_stream(const ShapeMap &shapes, int K, const std::vector<MixEntry> &stream, int32_t kind, int64_t sweeps,
                int32_t ex, uint64_t budget, double *rate) {
  const std::string sh = format_shapes(shapes);
  rfim_server_config sc{};
  sc.mem_budget_bytes = budget;
  sc.max_slots = (int32_t)stream.size();
  sc.intervals_per_launch = K;
  sc.batch_shapes = sh.c_str();
  rfim_server *s = nullptr;
  int rc = rfim_server_create(&sc, &s);
  if (rc != RFIM_OK) return rc;
  *rate = 0.0;
  for (int pass = 0; pass < 2 && rc == RFIM_OK; ++pass) {
    std::vector<uint64_t> tickets;
    double attempts = 0.0;
    const Clock::time_point t0 = Clock::now();
    for (size_t i = 0; i < stream.size() && rc == RFIM_OK; ++i) {
      const int L = stream[i].L, R = stream[i].R;
      std::vector<double> T(R);
      for (int k = 0; k < R; ++k) T[k] = std::pow(5.0, (double)k / (double)(R - 1));  // geometric in [1, 5]
      rfim_config c{};
      c.L = L;
      c.R = R;
      c.R_capacity = R;
      c.J = 1.0f;
      c.h = 1.0f;
      c.field_kind = kind;
      c.field_seed = 1u + (uint32_t)i;
      c.seed = 42u;
      c.realization = (uint32_t)i;
      c.temps = T.data();
      c.layout = RFIM_LAYOUT_BITPACK;
      uint64_t tk = 0;
      rc = rfim_server_submit(s, &c, sweeps, ex, sweeps / ex / 2, &tk);
      tickets.push_back(tk);
      attempts += (double)L * L * L * R * (double)sweeps;
    }
    for (size_t i = 0; i < tickets.size() && rc == RFIM_OK; ++i) {
      while ((rc = rfim_server_poll(s, tickets[i], nullptr, nullptr)) == RFIM_EBUSY)
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    const double dt = seconds(t0, Clock::now());
    if (rc == RFIM_OK && pass == 1) *rate = attempts / (dt * 1e9);
  }
  if (rc != RFIM_OK) g_server_error = std::string("tuning stream: ") + rfim_server_last_error(s);
  rfim_server_destroy(s);
  return rc;
}

// The entries repeated until their work items (at replicas per item g_min) fill `items` CTAs.
std::vector<MixEntry> fill_stream(const std::vector<MixEntry> &base, int g_min, int items) {
  std::vector<MixEntry> out;
  int have = 0;
  while (have < items || out.size() < base.size()) {
    const MixEntry &e = base[out.size() % base.size()];
    out.push_back(e);
    have += (e.R + g_min - 1) / g_min;
  }
  return out;
}

std::vector<BatchShape> shape_candidates(int L) {
  switch (L) {
    case 64: return {{2, 2}, {4, 2}, {2, 1}, {4, 1}, {1, 1}};
    case 32: return {{8, 2}, {4, 2}, {16, 2}, {4, 1}, {8, 1}};
    case 16: return {{16, 1}, {8, 1}, {32, 1}, {4, 1}};
    default: return {{16, 1}, {32, 1}, {64, 1}, {8, 1}};
  }
}

}  // namespace

extern "C" int rfim_server_tune(const rfim_server_tune_config *t, char *shapes_out, int32_t cap, int32_t *intervals_out,
                                double *attempts_per_ns) {
  if (!t || t->n < 1 || !t->L || !t->R || t->exchange_every < 1 || t->sweeps < t->exchange_every ||
      t->sweeps % t->exchange_every || t->mem_budget_bytes < (1u << 20) ||
      !(t->field_kind == RFIM_FIELD_BIMODAL || t->field_kind == RFIM_FIELD_GAUSSIAN))
    return server_fail(nullptr, RFIM_EINVAL, "rfim_server_tune: invalid configuration");
  std::vector<MixEntry> mix;
  for (int32_t i = 0; i < t->n; ++i) {
    if (!bits_supported(t->L[i]) || t->R[i] < 2 || t->R[i] > kMaxServedR)
      return server_fail(nullptr, RFIM_EINVAL, "rfim_server_tune: L must be 8, 16, 32 or 64 and R in [2, 1024]");
    mix.push_back({t->L[i], t->R[i]});
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  ShapeMap best = default_shapes();
  for (int L : {64, 32, 16, 8}) {
    std::vector<MixEntry> of_L;
    for (const MixEntry &e : mix)
      if (e.L == L) of_L.push_back(e);
    if (of_L.empty()) continue;
    int g_max = 1;
    for (const BatchShape &c : shape_candidates(L)) g_max = std::max(g_max, c.G);
    const std::vector<MixEntry> stream = fill_stream(of_L, g_max, 2 * sms);
    double best_rate = -1.0;
    for (const BatchShape &c : shape_candidates(L)) {
      if (!shape_ok(L, c.G, c.GT)) continue;
      ShapeMap m = best;
      m[L] = c;
      double r = 0.0;
      const int rc = time_stream(m, 4, stream, t->field_kind, t->sweeps, t->exchange_every, t->mem_budget_bytes, &r);
      if (rc != RFIM_OK) return rc;
      if (r > best_rate) {
        best_rate = r;
        best[L] = c;
      }
    }
  }
  int g_max = 1;
  for (const auto &kv : best) g_max = std::max(g_max, kv.second.G);
  const std::vector<MixEntry> stream = fill_stream(mix, g_max, 2 * sms);
  int best_k = 4;
  double best_rate = -1.0;
  for (int K : {1, 2, 4, 8}) {
    double r = 0.0;
    const int rc = time_stream(best, K, stream, t->field_kind, t->sweeps, t->exchange_every, t->mem_budget_bytes, &r);
    if (rc != RFIM_OK) return rc;
    if (r > best_rate) {
      best_rate = r;
      best_k = K;
    }
  }
  const std::string text = format_shapes(best);
  {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    g_tuned_shapes = text;
    g_tuned_intervals = best_k;
  }
  if (shapes_out && cap > 0) snprintf(shapes_out, (size_t)cap, "%s", text.c_str());
  if (intervals_out) *intervals_out = best_k;
  if (attempts_per_ns) *attempts_per_ns = best_rate;
  return RFIM_OK;
}
