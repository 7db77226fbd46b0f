/*
 * rfim.h -- C ABI of librfim: Exchange Monte Carlo (parallel tempering) for the 3D Random Field
 * Ising Model on one GB300 GPU.
 *
 * Paper: C. A. Navarro, W. Huang, Y. Deng, "Adaptive Multi-GPU Exchange Monte Carlo for the 3D
 * Random Field Ising Model".  Passages implemented behind this interface:
 *   Eq. 1      Hamiltonian H = -J sum_<ij> s_i s_j - h sum_i h_i s_i, periodic L^3 lattice.
 *   Sec. 3.1   steps 1-4: temperature set, one field realization shared by all replicas, random
 *              start, p Metropolis sweeps between exchanges of odd xor even adjacent pairs.
 *   Eq. 2      exchange probability, read as W = min(1, e^Delta),
 *              Delta = (beta_k - beta_k+1)(E(X_k) - E(X_k+1)).
 *   Eq. 3      alternator A = (x + y + z) mod 2: colour 0 sites, then colour 1 sites.
 *   Sec. 3.3   temperatures are swapped, not lattices ("trs"/"rts" index arrays).
 *   Sec. 4     adaptive temperature set: midpoint insertion in the a lowest-rate intervals.
 *   Sec. 7     Eqs. 11-12: per-temperature sums of e, e^2, |m|, m^2, m^4 (one per exchange step).
 *
 * Conventions
 *   - Every function returns RFIM_OK (0) or a negative RFIM_E* code; nothing throws across the ABI.
 *     rfim_last_error(ctx) returns the message of the last failure on that context.
 *   - A context owns all device memory it allocates (cudaMalloc in rfim_create, freed in
 *     rfim_destroy).  The CUDA stream in rfim_config is borrowed and must outlive the context;
 *     NULL means the legacy default stream.  The device is the one current at rfim_create.
 *   - Host pointers passed in are copied before the call returns.  Work is enqueued
 *     asynchronously on the context's stream; functions that return host data synchronise it.
 *   - A context is not thread safe; distinct contexts may be used from distinct threads.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), keyed and counted so that every flip and
 * exchange decision is reproducible (the paper names no generator):
 *   c3(tag, stage, colour) = (tag << 28) | (stage << 1) | colour;  tags INIT 1, METRO 2, EXCH 3, FIELD 4
 *   field bimodal : key (field_seed, realization), ctr (i>>2, 0, 0, c3(FIELD,0,0)), word i&3, top bit 0 -> +1
 *   field gaussian: key (field_seed, realization), ctr (i>>1, 1, 0, c3(FIELD,0,0)), words 2(i&1), 2(i&1)+1,
 *                   Box-Muller in double, rounded to float
 *   init          : key (seed, realization), ctr (i>>2, r, 0, c3(INIT,stage,0)), word i&3, top bit 0 -> +1
 *   metropolis    : key (seed, realization), ctr (q>>2, r, sweep, c3(METRO,stage,colour)), word q&3,
 *                   q = (x>>1) + (L/2)(y + L z)  (index of a site within its colour)
 *   exchange      : key (seed, realization), ctr (k, 0, j, c3(EXCH,stage,0)), word 0
 * Site index i = x + L (y + L z); replica index r names a lattice (it keeps its index when
 * temperatures are exchanged); temperature index k orders the ascending temperature set.
 */
#ifndef RFIM_H_
#define RFIM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RFIM_OK 0
#define RFIM_EINVAL (-1)   /* invalid argument or configuration */
#define RFIM_ENOMEM (-2)   /* device or host allocation failed */
#define RFIM_ECUDA (-3)    /* a CUDA call failed (message in rfim_last_error) */
#define RFIM_ETIMEOUT (-4) /* a bounded device-side wait expired */
#define RFIM_EBUSY (-5)    /* result not ready yet (serving poll) */
#define RFIM_ESTATE (-6)   /* call not valid in the current state */
#define RFIM_EBOUNDS (-7)  /* a device bounds check failed (debug build librfim_debug.so only) */

/* field kinds (Sec. 3.1 step 2 uses the bimodal field) */
#define RFIM_FIELD_BIMODAL 0  /* h_i = +-1 equiprobable, drawn from field_seed */
#define RFIM_FIELD_GAUSSIAN 1 /* h_i ~ N(0,1), drawn from field_seed */
#define RFIM_FIELD_EXPLICIT 2 /* h_i given by the caller (float[L^3], unscaled); float arithmetic */

/* spin storage layouts on the device; both give bit-identical trajectories */
#define RFIM_LAYOUT_INT8 0    /* one byte per spin, any even L >= 2 */
#define RFIM_LAYOUT_BITPACK 1 /* one bit per spin, L in {8, 16, 32, 64} */

typedef struct rfim_ctx rfim_ctx;

typedef struct {
  int32_t L;             /* linear size, even, >= 2 (N = L^3 sites) */
  int32_t R;             /* number of temperature replicas, >= 2 */
  int32_t R_capacity;    /* >= R; device storage is sized for this many replicas so that the
                            adaptive temperature set (Sec. 4) can grow without reallocation */
  float J;               /* coupling */
  float h;               /* field strength; hh_i = (float)h * h_i in float */
  int32_t field_kind;    /* RFIM_FIELD_* */
  const float *field;    /* EXPLICIT only: host float[L^3] unscaled h_i, natural site order */
  uint32_t field_seed;   /* key word 0 of the field stream */
  uint32_t seed;         /* key word 0 of the dynamics streams */
  uint32_t realization;  /* key word 1 of all streams (disorder realization id) */
  const double *temps;   /* host double[R], strictly ascending, > 0 */
  int32_t layout;        /* RFIM_LAYOUT_* */
  void *stream;          /* cudaStream_t (borrowed) or NULL */
} rfim_config;

/* Creates a context: copies the temperature set and (EXPLICIT) the field, generates the field
   on the device otherwise, and draws the random start of stage 0 (Sec. 3.1 steps 1-3).
   Errors: RFIM_EINVAL for odd L, L < 2, R < 2, R > R_capacity, non-ascending or non-positive
   temperatures, an unknown kind/layout, a missing explicit field, or a layout that does not
   support L; RFIM_ENOMEM if device memory runs out (nothing leaks); RFIM_ECUDA otherwise. */
int rfim_create(const rfim_config *cfg, rfim_ctx **out);

/* Frees everything the context owns (synchronising its stream first).  NULL is accepted. */
int rfim_destroy(rfim_ctx *ctx);

/* n_sweeps >= 0 full checkerboard sweeps (Eq. 3 colour 0 then colour 1) of every replica at
   its current temperature (Sec. 3.1 step 4, Metropolis).  Asynchronous. */
int rfim_sweep(rfim_ctx *ctx, int64_t n_sweeps);

/* One exchange step j = current exchange counter (Eq. 2; pairs k = j mod 2, j mod 2 + 2, ...):
   computes every replica's energy (Eq. 1), takes the swap decisions, permutes the temperature
   index (Sec. 3.3), updates per-pair attempt/acceptance counts, and, when j >= measure_from,
   adds one measurement per temperature (Sec. 7).  Asynchronous. */
int rfim_exchange(rfim_ctx *ctx, int64_t measure_from);

/* n_sweeps sweeps with an exchange step after every sweep whose 1-based global sweep count is
   a multiple of exchange_every (exchange_every <= 0: no exchanges).  Measurements as in
   rfim_exchange.  Asynchronous; the whole hot path runs on the device. */
int rfim_run(rfim_ctx *ctx, int64_t n_sweeps, int32_t exchange_every, int64_t measure_from);

/* Adaptive temperature set (Sec. 4).  For trial t = 1..n_trials: a fresh random start at stage t
   with the current set, sweeps_per_trial sweeps with exchanges every exchange_every sweeps, then
   rate_k = acc_k / att_k (0 if att_k == 0) and the midpoint temperature is inserted into each of
   the inserts_per_trial intervals of lowest rate (min-heap order, ties to the lower k).
   Afterwards the context is reset to stage 0 (fresh random start, identity permutation, counters
   and accumulators zero) with the final set.  temps_out (host, capacity temps_cap) receives the
   final set and *R_out its size.  rates_out may be NULL or host double[n_trials * R_capacity]:
   row t-1 receives trial t's pair rates.  Synchronous.
   Errors: RFIM_EINVAL if R + n_trials * inserts_per_trial > R_capacity, inserts_per_trial > R-1
   at some trial, exchange_every <= 0 or temps_cap too small. */
int rfim_adapt_temps(rfim_ctx *ctx, int32_t n_trials, int64_t sweeps_per_trial, int32_t exchange_every,
                     int32_t inserts_per_trial, double *temps_out, int32_t temps_cap, int32_t *R_out,
                     double *rates_out);

/* Observables: caller-owned host arrays sized for R (= the context's current R); any pointer may
   be NULL.  sums[k] are over the n_meas measurements at temperature index k (Sec. 7):
   e = E/N, e^2, |m|, m^2, m^4 with m = M/N, and F, the structure factor of the correlation length
   (zeros unless rfim_set_measure_xi enabled it; in served results zeros unless the server measures
   it).  att/acc have
   R-1 entries (pair k, k+1).  Synchronous. */
typedef struct {
  int32_t R;        /* out: current number of replicas */
  double *T;        /* [R] temperatures */
  double *e, *e2, *absm, *m2, *m4; /* [R] sums */
  uint64_t *att, *acc;             /* [R-1] */
  int64_t n_meas;   /* out */
  double *F;        /* [R] sums of the structure factor F (see rfim_set_measure_xi) */
} rfim_obs;
int rfim_observables(rfim_ctx *ctx, rfim_obs *out);

/* Enables (on != 0) or disables the measurement of the structure factor that the correlation
   length of Sec. 7 needs, read with the spins s_i for the printed h_i:
   F = (F1 + F2) / (3 L^3), F1 = sum over the axes d of (sum_i s_i cos(K i_d))^2, F2 the same with
   sin, K = 2 pi / L.  When enabled, every measuring exchange step (j >= measure_from) adds each
   replica's F to the sum of its temperature index, one extra launch per step.  Enable it before the
   first measurement (RFIM_ESTATE otherwise); rfim_adapt_temps and restarts clear the sums with the
   other accumulators.  Synchronous. */
int rfim_set_measure_xi(rfim_ctx *ctx, int32_t on);

/* Multi-hit double 3D checkerboard (Sec. 3.2; the multi-hit runs of Sec. 6) for the following
   sweeps, or (mh = 0) the plain checkerboard again.  The lattice is cut into tiles of tile^3
   sites, coarse colour (x/tile + y/tile + z/tile) mod 2; one sweep visits the tiles of coarse
   colour 0, then those of colour 1, and each visit makes mh black-white passes (fine colour 0,
   then 1) over the visited tiles with the neighbouring tiles frozen: every site is attempted mh
   times per sweep.  Pass h of sweep s draws the Philox words of counter
   (q >> 2, r, s mh + h mod 2^32, c3(METRO, stage, fine colour)), so counters repeat after
   2^32 / mh sweeps.  The paper keeps mh = 0 for its physics results; the multi-hit chain has the
   same Boltzmann law but other dynamics.  Bit layout only; tile in {8, 16, 32}, L in {16, 32, 64}
   divisible by 2 tile.  When the current launch shape has no multi-hit kernel (the grid-wide plan
   of L = 64) the context switches to the default cluster shape of its L (synchronous in that
   case).  Errors: RFIM_EINVAL (mh < 0, int8 layout, unsupported tile), RFIM_ENOMEM / RFIM_ECUDA
   from the plan switch. */
int rfim_set_multihit(rfim_ctx *ctx, int32_t mh, int32_t tile);

/* Thermal averages of one realization (Sec. 7) from its accumulators (obs as filled by
   rfim_observables or rfim_server_poll; T, e, e2, absm, m2, m4 required, F optional), for a lattice
   of N = L^3 sites.  out: host double[R][7] per temperature index k:
   <e>, C = (N / T_k^2)(<e^2> - <e>^2) (e the energy per site, the printed L^3 prefactor),
   <|m|>, <m^2>, <m^4>, <F>, xi = sqrt(N <m^2> / <F> - 1) (the printed <M^2> taken as the
   zero-wave-number structure factor N <m^2>, which has F's normalisation; no 1/(2 sin(K/2))
   factor, as printed; +infinity when <F> < 1e-20, i.e. a uniform lattice at every measurement).
   NaN where undefined (no measurements, no F, negative radicand).
   Host only; RFIM_EINVAL for missing arrays or N < 1. */
int rfim_thermal(const rfim_obs *obs, int32_t N, double *out);

/* Disorder average [.] of Sec. 7 over n realizations that share one temperature set: thermals is
   host double[n][R][7] (rfim_thermal's rows, realization-major), out host double[R][5] per
   temperature index: [<e>], [C], [<|m|>], [xi], and the Binder factor
   [g] = (3 - [<m^4>] / [<m^2>]^2) / 2 (a disorder-level average, as printed).  Host only. */
int rfim_disorder_average(const double *thermals, int32_t n, int32_t R, double *out);

/* State access for tests and checkpoint/resume.  spins: host int8[R][L^3] values +-1 in natural
   site order, indexed by replica r; t2r: int32[R] replica at temperature k; E: double[R] energy of
   each replica recomputed from the current spins (Eq. 1); any pointer may be NULL.  Synchronous. */
int rfim_get_state(rfim_ctx *ctx, int8_t *spins, int32_t *t2r, double *E, int64_t *sweep, int64_t *xstep);
/* Overwrites spins (int8[R][L^3], +-1; NULL keeps them), the permutation (t2r, NULL keeps it) and
   the sweep / exchange counters.  Accumulators and exchange statistics are left unchanged.
   Errors: RFIM_EINVAL if t2r is not a permutation or a spin is not +-1.  Synchronous. */
int rfim_set_state(rfim_ctx *ctx, const int8_t *spins, const int32_t *t2r, int64_t sweep, int64_t xstep);

/* Copies the unscaled field h_i (float[L^3], natural order) the context uses.  Synchronous. */
int rfim_get_field(rfim_ctx *ctx, float *h_out);

/* Message of the last failed call on ctx (or of the last failed rfim_create when ctx is NULL). */
const char *rfim_last_error(const rfim_ctx *ctx);

/* Number of kernel launches this context has enqueued since creation. */
int64_t rfim_launch_count(const rfim_ctx *ctx);

/* ---- Serving: continuous batching of independent disorder realizations -------------------------
   The quenched average (Sec. 7) needs many independent realizations.  A server owns a device
   memory arena and a worker thread: submitted realizations are admitted in arrival order as slots
   and arena memory free up; all resident ones advance together, intervals_per_launch exchange
   intervals per replay of a captured CUDA graph of persistent batched kernels; finished ones are
   retired between replays and their observables kept until polled.  Each result is the same as
   the realization run alone through the server (nothing is shared between realizations).  The
   bit layout is used (L in {8, 16, 32, 64}, R <= 1024). */
typedef struct rfim_server rfim_server;
typedef struct {
  uint64_t mem_budget_bytes;    /* device arena for resident realizations (admission control) */
  int32_t max_slots;            /* realizations resident at the same time, >= 1 */
  int32_t intervals_per_launch; /* exchange intervals per graph replay, >= 1; 0: the value chosen by
                                   the last rfim_server_tune of this process, else 4 */
  int32_t measure_xi;           /* != 0: also accumulate the structure factor F (rfim_set_measure_xi)
                                   on every measuring exchange step, fused into the batched kernel */
  const char *batch_shapes;     /* "L:G:GT,...": replicas per work item G and per thread GT of the
                                   batched kernel for each listed L (copied); NULL: the shapes of
                                   the last rfim_server_tune of this process, else built-in ones */
} rfim_server_config;
typedef struct {
  int64_t queued, resident, completed, graph_launches;
  double busy_s;   /* seconds spent in graph replays */
  double attempts; /* spin-flip attempts of completed realizations */
  int32_t grid;    /* CTAs of the persistent batched kernel */
  int32_t intervals_per_launch;
  char batch_shapes[64]; /* the shapes in use, "L:G:GT,..." for L = 64, 32, 16, 8 */
} rfim_server_info;
/* Errors: RFIM_EINVAL (bad configuration), RFIM_ENOMEM (arena), RFIM_ECUDA. */
int rfim_server_create(const rfim_server_config *cfg, rfim_server **out);
/* Queues one realization (cfg as for rfim_create; cfg->layout and cfg->stream are ignored, host
   arrays are copied before return) for n_sweeps sweeps, a positive multiple of exchange_every,
   with measurements from exchange step measure_from on.  *ticket identifies it. */
int rfim_server_submit(rfim_server *s, const rfim_config *cfg, int64_t n_sweeps, int32_t exchange_every,
                       int64_t measure_from, uint64_t *ticket);
/* RFIM_EBUSY while queued or running; RFIM_OK once finished: fills out (caller-owned arrays sized
   for its R, any may be NULL) and *latency_s (seconds from submit to retirement), then forgets the
   ticket.  out->F is the structure-factor sum when the server measures it, else zeros.
   RFIM_EINVAL for an unknown ticket; RFIM_ENOMEM if the realization cannot fit. */
int rfim_server_poll(rfim_server *s, uint64_t ticket, rfim_obs *out, double *latency_s);
int rfim_server_stats(rfim_server *s, rfim_server_info *out);
/* Stops the worker (resident work is abandoned) and frees everything.  NULL is accepted. */
int rfim_server_destroy(rfim_server *s);
/* Tuner of the batched kernel (spec batching pattern; it stands in for the paper's choice
   of block shape by the cost model of Sec. 3.2, Eq. (S) and (dS), which is prior art for Kepler).
   For each L of the expected mix it times every instantiated (G, GT) shape -- replicas per work
   item and per thread -- on scratch realizations of that L (enough to fill the GPU twice,
   sweeps each, closed loop on a scratch server with the other L at their best shapes so far),
   then times intervals_per_launch in {1, 2, 4, 8} on the whole mix with the chosen shapes.
   Later rfim_server_create calls in this process with batch_shapes == NULL and
   intervals_per_launch == 0 use the result.  Shapes and intervals change the launch only, not
   the results: every served realization takes the same decisions and sums in the same order
   whatever they are.  shapes_out (optional, cap chars) receives "L:G:GT,...", *intervals_out
   (optional) the interval count, *attempts_per_ns (optional) the rate of the chosen setting.
   Synchronous; creates scratch servers of mem_budget_bytes.  Errors: RFIM_EINVAL, RFIM_ENOMEM,
   RFIM_ECUDA (message in rfim_server_last_error(NULL)). */
typedef struct {
  int32_t n;                 /* entries of the expected mix */
  const int32_t *L, *R;      /* their lattice sizes (8, 16, 32, 64) and replica counts (<= 1024) */
  int32_t field_kind;        /* RFIM_FIELD_BIMODAL or RFIM_FIELD_GAUSSIAN (seeded scratch fields) */
  int32_t exchange_every;
  int64_t sweeps;            /* per scratch realization, a positive multiple of exchange_every */
  uint64_t mem_budget_bytes; /* arena of each scratch server */
} rfim_server_tune_config;
int rfim_server_tune(const rfim_server_tune_config *t, char *shapes_out, int32_t cap, int32_t *intervals_out,
                     double *attempts_per_ns);
const char *rfim_server_last_error(const rfim_server *s);

/* ---- Exchange step without device allocation ------------------------------------------------------
   The paper has no counterpart to this entry point; it exists for callers that cannot allocate
   device memory: a framework or arena that owns all of the device memory, or a latency-critical
   loop in which cudaMalloc / cudaFree would synchronise the device.
   It computes every replica's energy (Eq. 1) from caller-owned buffers and takes exchange step j
   exactly as rfim_exchange does (Eq. 2, Sec. 3.3; measurement of Sec. 7 when j >= measure_from),
   enqueued on `stream`.  It allocates nothing: its scratch (partial sums per replica and z slab,
   and an arrival counter) is a file-scope device array of 512 KiB that every GPU loading the
   library holds until exit.  R times the number of z slabs must fit 16384 slots (RFIM_EINVAL
   otherwise, message in rfim_last_error(NULL)).  Every call looks up the array's address on the
   current device (cudaGetSymbolAddress, no stream work); its arrival counter is zero when the
   library loads and each call leaves it at zero.  All calls share the array, which keeps the last
   call's contents: calls that overlap on the GPU race and must not be issued.
   Buffers (all device pointers, caller-owned):
     spins : uint32[R][2][L^3/64] bit layout: for colour c = (x+y+z) mod 2 the site with
             q = (x>>1) + (L/2)(y + L z) is bit 8(q&3) + ((q&31)>>2) of word q>>5 (1 = up)
     field : float[L^3] unscaled h_i in natural order (bimodal: +-1, exact integer field term;
             otherwise float arithmetic on hh_i = (float)h * h_i)
     beta  : double[R] 1/T_k in ascending-temperature order
     t2r, r2t (int32[R], in/out), att, acc (uint64[R-1], in/out), obs (double[R][5], in/out),
     n_meas (int64, in/out), E (double[R], out), M (int64[R], out). */
typedef struct {
  int32_t L;           /* 8, 16, 32 or 64 */
  int32_t R;           /* >= 2 */
  float J, h;
  int32_t field_kind;  /* RFIM_FIELD_* */
  uint32_t seed, realization, stage;
  const uint32_t *spins;
  const float *field;
  const double *beta;
  int32_t *t2r, *r2t;
  uint64_t *att, *acc;
  double *obs;
  int64_t *n_meas;
  double *E;
  int64_t *M;
} rfim_exchange_buffers;
int rfim_exchange_noalloc(const rfim_exchange_buffers *b, uint32_t j, int64_t measure_from, void *stream);

/* Kernel timing.  rfim_profile(ctx, 1) clears earlier records and starts bracketing every
   sweep-kernel launch group (one rfim_sweep / exchange-interval worth of sweeps) and every
   energy + exchange pair with CUDA events on the context's stream; rfim_profile(ctx, 0) stops.
   rfim_profile_read synchronises the stream and returns the summed device time (ms) and the
   number of bracketed groups of each kind since the last rfim_profile call (a grid-wide launch
   that runs k exchange intervals counts k sweep groups).  Any output pointer may be NULL. */
int rfim_profile(rfim_ctx *ctx, int enable);
int rfim_profile_read(rfim_ctx *ctx, double *sweep_ms, int64_t *sweep_launches, double *exchange_ms,
                      int64_t *exchange_launches);

/* Launch-shape tuner for the bit layout.  Times every instantiated launch shape (cluster size S
   = z slabs per replica group, replicas G per cluster, replicas GT per thread, threads per CTA;
   S = 0 is the grid-wide cooperative plan with one CTA per SM, G replicas per (group, z plane)
   unit) on a scratch realization with this L, R and field kind (20-50 exchange intervals of 10
   sweeps each, CUDA-event timing) and remembers the fastest: later rfim_create calls in this
   process with the same L, R_capacity and field kind use it.  plan_out (optional, plan_cap chars)
   receives "S,G,GT,threads"; *attempts_per_ns (optional) the best rate.  Synchronous; allocates
   scratch realizations.  Errors: RFIM_EINVAL (unsupported L, R < 2), RFIM_ECUDA. */
int rfim_tune(int32_t L, int32_t R, int32_t field_kind, char *plan_out, int32_t plan_cap, double *attempts_per_ns);

/* Launch shape of this context's sweep kernel, in the format rfim_tune reports: "S,G,GT,threads"
   with ",4" appended when every word is split over four warps (S = 0: the grid-wide plan), and
   ",int8" appended when the int8 layout is staged as bits; "" when the context runs the int8
   kernels (L outside 8, 16, 32, 64).  plan_out receives at most plan_cap chars (NUL included).
   Errors: RFIM_EINVAL (NULL ctx or plan_out, plan_cap < 1). */
int rfim_get_plan(const rfim_ctx *ctx, char *plan_out, int32_t plan_cap);

/* Host-only self-check of the bit layout's word-level neighbour arithmetic (multi-spin coding,
   Eq. 3 colours) against direct neighbour lookup on a random L^3 lattice; needs no GPU.
   Returns the number of mismatching sites (0 = pass) or -1 for an unsupported L. */
int rfim_selftest_bits(int32_t L, uint32_t seed);

/* Host-only self-check of the partition used by the grid-wide bit-layout kernel (replica groups
   of 4 x z planes spread over P CTAs; other group sizes partition the same way): unique owners, pieces tiling every CTA's range.  Returns
   the number of violations (0 = pass) or -1 for invalid arguments. */
int rfim_selftest_grid(int32_t L, int32_t R, int32_t P);

/* Device self-test of the bounded waits that the grid-wide kernel uses between CTAs (the paper
   has no counterpart: its CTAs never wait on one another).  One thread waits for a progress word
   that nothing sets (set_flag = 0) or that is already set (set_flag = 1), for at most spin_limit
   polls (1 <= spin_limit <= 2^22, each poll followed by a 64 ns sleep).  Returns RFIM_ETIMEOUT when
   the wait expired (the kernel recorded it in its error word and returned), RFIM_OK when the flag
   was seen, RFIM_EINVAL for a bad spin_limit, RFIM_ECUDA on a CUDA error.  Synchronous on the
   default stream; the context of the calling thread stays usable after an expiry. */
int rfim_selftest_wait(int32_t spin_limit, int32_t set_flag);

/* Bounds-checked build (no counterpart in the paper; it stands in for a memory checker).  The same
   sources compiled with -DRFIM_DEBUG give librfim_debug.so (same C ABI; the Python binding loads it
   when RFIM_LIBRARY=debug).  In it the sweep kernels check the shared-memory lattice indices, the
   decision-table slots against the dynamic shared memory, the cluster peer ranks of the halo
   loads, the grid-wide partition (pieces, planes, owners, partial slots) and the no-alloc scratch
   slots; a failed check sets a bit of the launch's device error word and the access is skipped or
   redirected to a harmless index, so the kernel still ends normally (nothing traps).  The word is
   reported as RFIM_EBOUNDS by rfim_observables / rfim_get_state, by the server (fatal, at the next
   poll) and, after a synchronisation, by rfim_exchange_noalloc.  rfim_debug_build returns 1 in
   that library and 0 in librfim.so.  rfim_selftest_debug (debug library only; RFIM_ESTATE
   otherwise) runs one checked index that is out of range on purpose and returns RFIM_OK when the
   check caught it and the kernel finished, RFIM_EBOUNDS if it was not caught, RFIM_ECUDA on a CUDA
   error.  Synchronous on the default stream. */
int rfim_debug_build(void);
int rfim_selftest_debug(void);

#ifdef __cplusplus
}
#endif
#endif /* RFIM_H_ */
