/*
 * rfim_oracle.c -- plain, slow, single-threaded CPU oracle for the Exchange Monte Carlo
 * (parallel tempering) simulation of the 3D Random Field Ising Model.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
 * reference arm may load this library.  It shares no code, header, table or constant generator
 * with the CUDA path.  Built with -O2 -ffp-contract=off so that every float operation is
 * rounded on its own (no fused multiply-add), as the contract below requires.
 *
 * What it computes (paper: "Adaptive Multi-GPU Exchange Monte Carlo for the 3D Random Field
 * Ising Model", Navarro, Huang, Deng):
 *   - Eq. 1 (Hamiltonian): H = -J sum_<ij> s_i s_j - h sum_i h_i s_i on an L^3 periodic lattice.
 *   - Sec. 3.1 steps 1-4: M temperatures, one field realization shared by all replicas, random
 *     start, then repeated {Metropolis sweeps; exchange of odd xor even adjacent pairs}.
 *   - Eq. 2 (exchange probability), read as W = min(1, e^Delta), Delta = (b_k - b_k+1)(E_a - E_b).
 *   - Eq. 3 (alternator A = (x+y+z) mod 2): plain checkerboard, colour 0 then colour 1.
 *   - Sec. 3.3: temperatures are swapped, not lattices (t2r = "trs", r2t = "rts").
 *   - Sec. 4: adaptive temperature set, midpoint insertion at the a lowest exchange rates.
 *   - Sec. 7, Eqs. 11-12: per-temperature accumulators of e, e^2, |m|, m^2, m^4, and (when
 *     enabled) of the structure factor F of the correlation-length formula, with the spins s_i
 *     in place of the printed h_i: F = (F1 + F2) / (3 L^3), F1 = sum over the axes d of
 *     (sum_i s_i cos(K i_d))^2, F2 the same with sin, K = 2 pi / L.
 *
 * Random numbers (the paper names no generator): Philox4x32-10 from its published definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 *   word3 tag field c3(tag, stage, colour) = (tag << 28) | (stage << 1) | colour
 *   field  bimodal : key (field_seed, realization), ctr (i>>2, 0, 0, c3(FIELD,0,0)), word i&3,
 *                    h_i = +1 if the word's top bit is 0 else -1
 *   field  gaussian: key (field_seed, realization), ctr (i>>1, 1, 0, c3(FIELD,0,0)),
 *                    words 2(i&1), 2(i&1)+1 -> Box-Muller in double -> float
 *   init           : key (seed, realization), ctr (i>>2, r, 0, c3(INIT,stage,0)), word i&3,
 *                    s = +1 if top bit is 0 else -1
 *   metropolis     : key (seed, realization), ctr (q>>2, r, sweep, c3(METRO,stage,colour)), word q&3
 *                    with q = (x>>1) + (L/2)(y + L z) the index of the site within its colour
 *   exchange       : key (seed, realization), ctr (k, 0, j, c3(EXCH,stage,0)), word 0
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_TAG_INIT 1u
#define ORC_TAG_METRO 2u
#define ORC_TAG_EXCH 3u
#define ORC_TAG_FIELD 4u

#define ORC_FIELD_BIMODAL 0
#define ORC_FIELD_GAUSSIAN 1
#define ORC_FIELD_EXPLICIT 2

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. SC'11): S-box free Feistel-like rounds built from two 32x32->64  */
/* multiplications; the key is bumped by the Weyl constants between rounds.                    */
/* ------------------------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_W1 = 0xBB67AE85u; /* sqrt(3) - 1 */

void orc_philox4x32_10(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                       uint32_t out[4]) {
  uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3;
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static uint32_t tagword(uint32_t tag, uint32_t stage, uint32_t colour) {
  return (tag << 28) | (stage << 1) | colour;
}

/* ------------------------------------------------------------------------------------------ */
/* Field realization (Sec. 3.1 step 2; Eq. 1's h_i).                                            */
/* ------------------------------------------------------------------------------------------ */
/* Writes the unscaled field h_i (natural site order i = x + L(y + L z)). */
void orc_make_field(int32_t L, int32_t kind, uint32_t field_seed, uint32_t realization, float *h_out) {
  int64_t N = (int64_t)L * L * L;
  uint32_t w[4];
  for (int64_t i = 0; i < N; ++i) {
    if (kind == ORC_FIELD_BIMODAL) {
      orc_philox4x32_10(field_seed, realization, (uint32_t)(i >> 2), 0u, 0u, tagword(ORC_TAG_FIELD, 0, 0), w);
      uint32_t word = w[i & 3];
      h_out[i] = (word >> 31) ? -1.0f : 1.0f;
    } else {
      orc_philox4x32_10(field_seed, realization, (uint32_t)(i >> 1), 1u, 0u, tagword(ORC_TAG_FIELD, 0, 0), w);
      double u1 = ((double)w[2 * (i & 1)] + 0.5) * 0x1p-32;
      double u2 = ((double)w[2 * (i & 1) + 1] + 0.5) * 0x1p-32;
      double z = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
      h_out[i] = (float)z;
    }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Simulation state of one disorder realization with R temperature replicas.                   */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int32_t L, N, R, Rcap;
  float J, h;
  int32_t field_kind;
  uint32_t field_seed, seed, realization, stage;
  double *T;       /* [Rcap] ascending temperatures, T[k] belongs to temperature index k */
  float *hraw;     /* [N] unscaled field h_i */
  float *hh;       /* [N] hh_i = (float)h * h_i */
  int8_t *s;       /* [Rcap][N] spins +-1, natural site order, indexed by replica (lattice) r */
  int32_t *t2r;    /* [Rcap] replica holding temperature k ("trs" of Sec. 3.3) */
  int32_t *r2t;    /* [Rcap] temperature index of replica r ("rts") */
  uint64_t *att, *acc; /* [Rcap-1] exchange attempts / acceptances of pair (k, k+1) */
  double *E;       /* [Rcap] energy of replica r at the last exchange step */
  int64_t *M;      /* [Rcap] magnetisation sum of replica r at the last exchange step */
  double *obs;     /* [Rcap][5] sums of e, e^2, |m|, m^2, m^4 per temperature index */
  double *obsF;    /* [Rcap] sums of the structure factor F per temperature index */
  int32_t measure_xi;
  int32_t mh, tile; /* multi-hit double checkerboard: mh local passes per tile visit (0: off), tile edge */
  int64_t n_meas;
  int64_t sweep;   /* global sweep counter (0-based) */
  int64_t xstep;   /* global exchange step counter j (0-based) */
  /* bimodal acceptance thresholds per temperature: [k][sn+6 (0..12 even)][sh (0:-1,1:+1)] */
  uint64_t *thr;
} orc_t;

static int64_t site_index(int32_t L, int32_t x, int32_t y, int32_t z) {
  return (int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * z);
}

/* Sum of the six periodic nearest neighbours of site (x,y,z) of replica r (Eq. 1's <ij>). */
static int32_t neighbour_sum(const orc_t *o, int32_t r, int32_t x, int32_t y, int32_t z) {
  int32_t L = o->L;
  const int8_t *s = o->s + (int64_t)r * o->N;
  int32_t xp = (x + 1) % L, xm = (x + L - 1) % L;
  int32_t yp = (y + 1) % L, ym = (y + L - 1) % L;
  int32_t zp = (z + 1) % L, zm = (z + L - 1) % L;
  return s[site_index(L, xp, y, z)] + s[site_index(L, xm, y, z)] + s[site_index(L, x, yp, z)] +
         s[site_index(L, x, ym, z)] + s[site_index(L, x, y, zp)] + s[site_index(L, x, y, zm)];
}

/* Bimodal acceptance threshold for an energy change dE at inverse temperature beta:
   accept iff dE <= 0, else iff w < floor(exp(-beta dE) 2^32) clamped to [1, 2^32 - 1]. */
static uint64_t bimodal_threshold(double beta, double dE) {
  if (dE <= 0.0) return 0x100000000ull;
  double p = exp(-beta * dE) * 4294967296.0;
  double f = floor(p);
  if (f < 1.0) f = 1.0;
  if (f > 4294967295.0) f = 4294967295.0;
  return (uint64_t)f;
}

static void rebuild_thresholds(orc_t *o) {
  for (int32_t k = 0; k < o->R; ++k) {
    double beta = 1.0 / o->T[k];
    for (int32_t sn = -6; sn <= 6; sn += 2) {
      for (int32_t sh = 0; sh < 2; ++sh) {
        double shv = sh ? 1.0 : -1.0;
        /* dE = 2 (J s n + h s h_i), Eq. 1 differentiated w.r.t. one spin flip */
        double dE = 2.0 * ((double)o->J * (double)sn + (double)o->h * shv);
        o->thr[(int64_t)k * 26 + (sn + 6) * 2 + sh] = bimodal_threshold(beta, dE);
      }
    }
  }
}

void orc_destroy(orc_t *o) {
  if (!o) return;
  free(o->T); free(o->hraw); free(o->hh); free(o->s); free(o->t2r); free(o->r2t);
  free(o->att); free(o->acc); free(o->E); free(o->M); free(o->obs); free(o->obsF); free(o->thr);
  free(o);
}

/* Creates a realization.  field: NULL unless kind == EXPLICIT (then N unscaled floats).
   temps: R ascending temperatures.  Returns NULL on invalid input. */
orc_t *orc_create(int32_t L, int32_t R, int32_t Rcap, float J, float h, int32_t field_kind,
                  const float *field, uint32_t field_seed, uint32_t seed, uint32_t realization,
                  const double *temps) {
  if (L < 2 || (L & 1) || R < 2 || Rcap < R) return NULL;
  for (int32_t k = 0; k < R; ++k) {
    if (!(temps[k] > 0.0)) return NULL;
    if (k > 0 && !(temps[k] > temps[k - 1])) return NULL;
  }
  orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
  o->L = L; o->N = L * L * L; o->R = R; o->Rcap = Rcap; o->J = J; o->h = h;
  o->field_kind = field_kind; o->field_seed = field_seed; o->seed = seed; o->realization = realization;
  o->stage = 0;
  int64_t N = o->N;
  o->T = (double *)calloc(Rcap, sizeof(double));
  o->hraw = (float *)calloc(N, sizeof(float));
  o->hh = (float *)calloc(N, sizeof(float));
  o->s = (int8_t *)calloc((size_t)Rcap * N, 1);
  o->t2r = (int32_t *)calloc(Rcap, sizeof(int32_t));
  o->r2t = (int32_t *)calloc(Rcap, sizeof(int32_t));
  o->att = (uint64_t *)calloc(Rcap, sizeof(uint64_t));
  o->acc = (uint64_t *)calloc(Rcap, sizeof(uint64_t));
  o->E = (double *)calloc(Rcap, sizeof(double));
  o->M = (int64_t *)calloc(Rcap, sizeof(int64_t));
  o->obs = (double *)calloc((size_t)Rcap * 5, sizeof(double));
  o->obsF = (double *)calloc((size_t)Rcap, sizeof(double));
  o->thr = (uint64_t *)calloc((size_t)Rcap * 26, sizeof(uint64_t));
  memcpy(o->T, temps, sizeof(double) * R);
  if (field_kind == ORC_FIELD_EXPLICIT) {
    memcpy(o->hraw, field, sizeof(float) * N);
  } else {
    orc_make_field(L, field_kind, field_seed, realization, o->hraw);
  }
  for (int64_t i = 0; i < N; ++i) o->hh[i] = h * o->hraw[i];
  rebuild_thresholds(o);
  return o;
}

/* Random start (Sec. 3.1 step 3) for replicas 0..R-1 at the given stage; resets the
   permutation to the identity and all counters and accumulators. */
void orc_reset(orc_t *o, uint32_t stage) {
  o->stage = stage;
  uint32_t w[4];
  for (int32_t r = 0; r < o->R; ++r) {
    for (int64_t i = 0; i < o->N; ++i) {
      orc_philox4x32_10(o->seed, o->realization, (uint32_t)(i >> 2), (uint32_t)r, 0u,
                        tagword(ORC_TAG_INIT, stage, 0), w);
      o->s[(int64_t)r * o->N + i] = (w[i & 3] >> 31) ? -1 : 1;
    }
  }
  for (int32_t k = 0; k < o->Rcap; ++k) {
    o->t2r[k] = k; o->r2t[k] = k; o->att[k] = 0; o->acc[k] = 0; o->E[k] = 0.0; o->M[k] = 0;
  }
  memset(o->obs, 0, sizeof(double) * 5 * o->Rcap);
  memset(o->obsF, 0, sizeof(double) * o->Rcap);
  o->n_meas = 0; o->sweep = 0; o->xstep = 0;
}

/* Energy change of flipping site i of replica r (Eq. 1), float path used for Gaussian and
   explicit fields: f = J*n + hh_i in float (two roundings), dE = 2 s_i f (exact). */
static float delta_e_float(const orc_t *o, int32_t r, int32_t x, int32_t y, int32_t z) {
  int64_t i = site_index(o->L, x, y, z);
  int32_t n = neighbour_sum(o, r, x, y, z);
  float Jn = o->J * (float)n;
  float f = Jn + o->hh[i];
  float si = (float)o->s[(int64_t)r * o->N + i];
  return 2.0f * si * f;
}

/* Energy change in double for the bimodal path: dE = 2 (J s n + h s h_i). */
static double delta_e_bimodal(const orc_t *o, int32_t r, int32_t x, int32_t y, int32_t z) {
  int64_t i = site_index(o->L, x, y, z);
  int32_t n = neighbour_sum(o, r, x, y, z);
  int32_t si = o->s[(int64_t)r * o->N + i];
  double shv = (double)(si * (int32_t)o->hraw[i]);
  return 2.0 * ((double)o->J * (double)(si * n) + (double)o->h * shv);
}

/* Exposed for tests: single-flip energy change of site (x,y,z) of replica r as the sweep uses it. */
double orc_delta_e(const orc_t *o, int32_t r, int32_t x, int32_t y, int32_t z) {
  if (o->field_kind == ORC_FIELD_BIMODAL) return delta_e_bimodal(o, r, x, y, z);
  return (double)delta_e_float(o, r, x, y, z);
}

/* Metropolis update (Sec. 3.1 step 4) of site (x,y,z) of replica r at temperature index k with
   the random word `word`: accept iff dE <= 0 or the word passes the Boltzmann test, then flip. */
static void metropolis_site(orc_t *o, int32_t r, int32_t k, int32_t x, int32_t y, int32_t z, uint32_t word) {
  int64_t i = site_index(o->L, x, y, z);
  int accept;
  if (o->field_kind == ORC_FIELD_BIMODAL) {
    int32_t si = o->s[(int64_t)r * o->N + i];
    int32_t n = neighbour_sum(o, r, x, y, z);
    int32_t sn = si * n;
    int32_t sh = (si * (int32_t)o->hraw[i]) > 0 ? 1 : 0;
    uint64_t thr = o->thr[(int64_t)k * 26 + (sn + 6) * 2 + sh];
    accept = (uint64_t)word < thr;
  } else {
    float betaf = (float)(1.0 / o->T[k]);
    float dE = delta_e_float(o, r, x, y, z);
    float xarg = betaf * dE;
    double u = (double)(word >> 8) * 0x1p-24;
    accept = (dE <= 0.0f) || (u < exp(-(double)xarg));
  }
  if (accept) o->s[(int64_t)r * o->N + i] = (int8_t)(-o->s[(int64_t)r * o->N + i]);
}

/* One pass over the sites of colour `colour` (Eq. 3) of every replica, with the Philox counter
   (q >> 2, r, c2, c3(METRO, stage, colour)), word q & 3, for the site q of the colour.  With
   tile > 0 only the sites in tiles of coarse colour `coarse` are visited (double checkerboard). */
static void colour_pass(orc_t *o, int32_t colour, uint32_t c2, int32_t tile, int32_t coarse) {
  int32_t L = o->L, Lh = L / 2;
  int64_t half = (int64_t)o->N / 2;
  uint32_t w[4];
  for (int32_t r = 0; r < o->R; ++r) {
    int32_t k = o->r2t[r];
    int64_t cached = -1;
    for (int64_t q = 0; q < half; ++q) {
      int32_t xh = (int32_t)(q % Lh);
      int32_t y = (int32_t)((q / Lh) % L);
      int32_t z = (int32_t)(q / ((int64_t)Lh * L));
      int32_t x = 2 * xh + ((colour + y + z) & 1);
      if (tile > 0 && ((x / tile + y / tile + z / tile) & 1) != coarse) continue;
      if ((q >> 2) != cached) {
        orc_philox4x32_10(o->seed, o->realization, (uint32_t)(q >> 2), (uint32_t)r, c2,
                          tagword(ORC_TAG_METRO, o->stage, (uint32_t)colour), w);
        cached = q >> 2;
      }
      metropolis_site(o, r, k, x, y, z, w[q & 3]);
    }
  }
}

/* One sweep of every replica.  Plain checkerboard (Eq. 3, Sec. 3.1 step 4): all colour-0 sites,
   then all colour-1 sites, counter word 2 = the sweep.  Multi-hit double 3D checkerboard (Sec. 3.2;
   the multi-hit runs of Sec. 6): the lattice is cut into tiles of tile^3 sites with coarse colour
   (x/tile + y/tile + z/tile) mod 2; the tiles of coarse colour 0 are visited, then those of
   coarse colour 1, and a visit makes mh local passes, each a black-white pass (fine colour 0,
   then 1) over the visited tiles with the neighbouring tiles frozen.  Pass h of sweep s uses
   counter word 2 = s * mh + h (mod 2^32), so every site draws a fresh word at each hit. */
void orc_sweep(orc_t *o) {
  uint32_t sweep = (uint32_t)o->sweep;
  if (o->mh > 0) {
    for (int32_t coarse = 0; coarse < 2; ++coarse)
      for (int32_t h = 0; h < o->mh; ++h)
        for (int32_t colour = 0; colour < 2; ++colour)
          colour_pass(o, colour, sweep * (uint32_t)o->mh + (uint32_t)h, o->tile, coarse);
  } else {
    for (int32_t colour = 0; colour < 2; ++colour) colour_pass(o, colour, sweep, 0, 0);
  }
  o->sweep += 1;
}

/* Selects the multi-hit double checkerboard (mh >= 1 local passes per tile visit, tiles of edge
   tile with L divisible by 2 tile, so that the coarse colouring is periodic) or, with mh = 0,
   the plain checkerboard.  Returns 0, or -1 for an invalid tile. */
int32_t orc_set_multihit(orc_t *o, int32_t mh, int32_t tile) {
  if (mh < 0) return -1;
  if (mh > 0 && (tile < 1 || o->L % (2 * tile) != 0)) return -1;
  o->mh = mh;
  o->tile = mh > 0 ? tile : 0;
  return 0;
}

/* Energy of replica r (Eq. 1): E = -J B - F with B summed over the 3N forward bonds. */
double orc_energy(const orc_t *o, int32_t r, int64_t *B_out, double *F_out, int64_t *M_out) {
  int32_t L = o->L;
  const int8_t *s = o->s + (int64_t)r * o->N;
  int64_t B = 0, M = 0, Fi = 0;
  double F = 0.0;
  for (int32_t z = 0; z < L; ++z)
    for (int32_t y = 0; y < L; ++y)
      for (int32_t x = 0; x < L; ++x) {
        int64_t i = site_index(L, x, y, z);
        int32_t si = s[i];
        B += si * (s[site_index(L, (x + 1) % L, y, z)] + s[site_index(L, x, (y + 1) % L, z)] +
                   s[site_index(L, x, y, (z + 1) % L)]);
        M += si;
        if (o->field_kind == ORC_FIELD_BIMODAL) Fi += si * (int32_t)o->hraw[i];
        else F += (double)o->hh[i] * (double)si;
      }
  if (o->field_kind == ORC_FIELD_BIMODAL) F = (double)o->h * (double)Fi;
  if (B_out) *B_out = B;
  if (F_out) *F_out = F;
  if (M_out) *M_out = M;
  return -(double)o->J * (double)B - F;
}

/* Structure factor of replica r at the smallest nonzero wave number (Sec. 7, correlation
   length; s_i read for the printed h_i): F = (F1 + F2) / (3 L^3) with F1 = sum over the three
   axes d of (sum_i s_i cos(K i_d))^2 and F2 the same with sin, K = 2 pi / L.  Direct sums over
   the sites in natural order, in double. */
double orc_structure_F(const orc_t *o, int32_t r) {
  const int32_t L = o->L;
  const double K = 2.0 * 3.14159265358979323846 / (double)L;
  const int8_t *s = o->s + (int64_t)r * o->N;
  double c[3] = {0.0, 0.0, 0.0}, sn[3] = {0.0, 0.0, 0.0};
  for (int32_t z = 0; z < L; ++z)
    for (int32_t y = 0; y < L; ++y)
      for (int32_t x = 0; x < L; ++x) {
        const double si = (double)s[site_index(L, x, y, z)];
        const int32_t xyz[3] = {x, y, z};
        for (int d = 0; d < 3; ++d) {
          c[d] += si * cos(K * (double)xyz[d]);
          sn[d] += si * sin(K * (double)xyz[d]);
        }
      }
  double F1 = 0.0, F2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    F1 += c[d] * c[d];
    F2 += sn[d] * sn[d];
  }
  return (F1 + F2) / (3.0 * (double)o->N);
}

void orc_set_measure_xi(orc_t *o, int32_t on) { o->measure_xi = on ? 1 : 0; }

/* One exchange step j (Eq. 2 with W = min(1, e^Delta); pairs k = j mod 2, j mod 2 + 2, ...,
   temperatures swapped through t2r / r2t as in Sec. 3.3), then the measurement of Sec. 7
   when j >= measure_from. */
void orc_exchange(orc_t *o, int64_t measure_from) {
  for (int32_t r = 0; r < o->R; ++r) o->E[r] = orc_energy(o, r, NULL, NULL, &o->M[r]);
  uint32_t j = (uint32_t)o->xstep;
  uint32_t w[4];
  for (int32_t k = (int32_t)(j & 1u); k + 1 < o->R; k += 2) {
    int32_t a = o->t2r[k], b = o->t2r[k + 1];
    double bk = 1.0 / o->T[k], bk1 = 1.0 / o->T[k + 1];
    double delta = (bk - bk1) * (o->E[a] - o->E[b]);
    orc_philox4x32_10(o->seed, o->realization, (uint32_t)k, 0u, j, tagword(ORC_TAG_EXCH, o->stage, 0), w);
    double u = (double)w[0] * 0x1p-32;
    int accept = (delta >= 0.0) || (u < exp(delta));
    o->att[k] += 1;
    if (accept) {
      o->acc[k] += 1;
      o->t2r[k] = b; o->t2r[k + 1] = a;
      o->r2t[b] = k; o->r2t[a] = k + 1;
    }
  }
  if ((int64_t)j >= measure_from) {
    for (int32_t k = 0; k < o->R; ++k) {
      int32_t a = o->t2r[k];
      double e = o->E[a] / (double)o->N;
      double m = (double)o->M[a] / (double)o->N;
      double *acc = o->obs + (int64_t)k * 5;
      acc[0] += e; acc[1] += e * e; acc[2] += fabs(m); acc[3] += m * m; acc[4] += m * m * m * m;
      if (o->measure_xi) o->obsF[k] += orc_structure_F(o, a);
    }
    o->n_meas += 1;
  }
  o->xstep += 1;
}

/* Sweeps with an exchange step after every exchange_every-th sweep (global sweep count). */
void orc_run(orc_t *o, int64_t n_sweeps, int32_t exchange_every, int64_t measure_from) {
  for (int64_t t = 0; t < n_sweeps; ++t) {
    orc_sweep(o);
    if (exchange_every > 0 && (o->sweep % exchange_every) == 0) orc_exchange(o, measure_from);
  }
}

/* Lowest-rate selection of Sec. 4: a min-heap keyed by (rate, k); pops `a` entries. */
static int heap_less(const double *rate, const int32_t *idx, int32_t i, int32_t j) {
  if (rate[i] != rate[j]) return rate[i] < rate[j];
  return idx[i] < idx[j];
}
static void heap_sift_down(double *rate, int32_t *idx, int32_t n, int32_t i) {
  for (;;) {
    int32_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < n && heap_less(rate, idx, l, m)) m = l;
    if (r < n && heap_less(rate, idx, r, m)) m = r;
    if (m == i) return;
    double tr = rate[i]; rate[i] = rate[m]; rate[m] = tr;
    int32_t ti = idx[i]; idx[i] = idx[m]; idx[m] = ti;
    i = m;
  }
}
/* Picks the `a` pairs with the lowest rates; writes their pair indices (pop order) to out. */
void orc_select_lowest(const double *rates, int32_t npairs, int32_t a, int32_t *out) {
  double *hr = (double *)malloc(sizeof(double) * (npairs > 0 ? npairs : 1));
  int32_t *hi = (int32_t *)malloc(sizeof(int32_t) * (npairs > 0 ? npairs : 1));
  for (int32_t k = 0; k < npairs; ++k) { hr[k] = rates[k]; hi[k] = k; }
  for (int32_t i = npairs / 2 - 1; i >= 0; --i) heap_sift_down(hr, hi, npairs, i);
  int32_t n = npairs;
  for (int32_t t = 0; t < a && n > 0; ++t) {
    out[t] = hi[0];
    hr[0] = hr[n - 1]; hi[0] = hi[n - 1]; --n;
    heap_sift_down(hr, hi, n, 0);
  }
  free(hr); free(hi);
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* Adaptive temperatures (Sec. 4): n_trials fresh trial runs (stage t = 1..n_trials), each
   followed by the insertion of the midpoint temperature into the `inserts` lowest-rate
   intervals.  Afterwards the realization is reset to stage 0 with the final set.
   rates_out (optional): [n_trials][Rcap] per-trial rates of the pre-insertion pairs.
   Returns the final R, or -1 when R would exceed Rcap or an argument is invalid. */
int32_t orc_adapt(orc_t *o, int32_t n_trials, int64_t sweeps_per_trial, int32_t exchange_every,
                  int32_t inserts, double *rates_out) {
  if (n_trials < 0 || inserts < 0 || exchange_every <= 0) return -1;
  if (o->R + (int64_t)n_trials * inserts > o->Rcap) return -1;
  for (int32_t t = 1; t <= n_trials; ++t) {
    if (inserts > o->R - 1) return -1;
    rebuild_thresholds(o);
    orc_reset(o, (uint32_t)t);
    orc_run(o, sweeps_per_trial, exchange_every, INT64_MAX);
    int32_t np = o->R - 1;
    double *rates = (double *)malloc(sizeof(double) * np);
    for (int32_t k = 0; k < np; ++k) rates[k] = o->att[k] ? (double)o->acc[k] / (double)o->att[k] : 0.0;
    if (rates_out)
      for (int32_t k = 0; k < np; ++k) rates_out[(int64_t)(t - 1) * o->Rcap + k] = rates[k];
    int32_t *pick = (int32_t *)malloc(sizeof(int32_t) * (inserts > 0 ? inserts : 1));
    orc_select_lowest(rates, np, inserts, pick);
    int32_t R0 = o->R;
    for (int32_t t2 = 0; t2 < inserts; ++t2) {
      int32_t k = pick[t2];
      o->T[R0 + t2] = 0.5 * (o->T[k] + o->T[k + 1]);
    }
    o->R = R0 + inserts;
    qsort(o->T, (size_t)o->R, sizeof(double), cmp_double);
    free(rates); free(pick);
  }
  rebuild_thresholds(o);
  orc_reset(o, 0u);
  return o->R;
}

/* ---------------------------------- accessors for tests ---------------------------------- */
int32_t orc_R(const orc_t *o) { return o->R; }
int32_t orc_N(const orc_t *o) { return o->N; }
int64_t orc_sweep_count(const orc_t *o) { return o->sweep; }
int64_t orc_xstep_count(const orc_t *o) { return o->xstep; }
int64_t orc_n_meas(const orc_t *o) { return o->n_meas; }

void orc_get_temps(const orc_t *o, double *T) { memcpy(T, o->T, sizeof(double) * o->R); }
void orc_get_field(const orc_t *o, float *hraw, float *hh) {
  if (hraw) memcpy(hraw, o->hraw, sizeof(float) * o->N);
  if (hh) memcpy(hh, o->hh, sizeof(float) * o->N);
}
void orc_get_spins(const orc_t *o, int8_t *s) { memcpy(s, o->s, (size_t)o->R * o->N); }
void orc_set_spins(orc_t *o, const int8_t *s) { memcpy(o->s, s, (size_t)o->R * o->N); }
void orc_get_perm(const orc_t *o, int32_t *t2r, int32_t *r2t) {
  if (t2r) memcpy(t2r, o->t2r, sizeof(int32_t) * o->R);
  if (r2t) memcpy(r2t, o->r2t, sizeof(int32_t) * o->R);
}
void orc_set_perm(orc_t *o, const int32_t *t2r) {
  for (int32_t k = 0; k < o->R; ++k) { o->t2r[k] = t2r[k]; o->r2t[t2r[k]] = k; }
}
void orc_set_counters(orc_t *o, int64_t sweep, int64_t xstep) { o->sweep = sweep; o->xstep = xstep; }
void orc_get_exchange_stats(const orc_t *o, uint64_t *att, uint64_t *acc) {
  if (att) memcpy(att, o->att, sizeof(uint64_t) * (o->R - 1));
  if (acc) memcpy(acc, o->acc, sizeof(uint64_t) * (o->R - 1));
}
void orc_get_energies(const orc_t *o, double *E, int64_t *M) {
  if (E) memcpy(E, o->E, sizeof(double) * o->R);
  if (M) memcpy(M, o->M, sizeof(int64_t) * o->R);
}
void orc_get_obs(const orc_t *o, double *obs) { memcpy(obs, o->obs, sizeof(double) * 5 * o->R); }
void orc_get_obsF(const orc_t *o, double *F) { memcpy(F, o->obsF, sizeof(double) * o->R); }
/* Bimodal threshold used for an energy change dE at inverse temperature beta (tests). */
uint64_t orc_bimodal_threshold(double beta, double dE) { return bimodal_threshold(beta, dE); }
