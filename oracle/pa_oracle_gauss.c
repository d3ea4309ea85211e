/*
 * pa_oracle_gauss.c -- plain, slow CPU oracle for population annealing on
 * Ising spin glasses with Gaussian couplings (the model of the paper's
 * Sec. 4: couplings drawn from a Gaussian of mean zero and variance one).
 *
 * TEST INFRASTRUCTURE ONLY: it checks the CUDA path and is never linked into
 * the product library.  Built with -ffp-contract=off.
 *
 * Couplings are fixed-point integers J_q (physical J = J_q * 2^-15), so
 * energies and energy changes are exact integers and no summation order can
 * change a result.  The Metropolis test at a rise dE_q > 0 uses the top 24
 * bits u24 of the site's uniform: accept iff (float)u24 < fexp(x) * 2^24 with
 * x = -(float(beta') * float(dE_q)) * 2^-15 in single precision; fexp is a
 * deterministic single-precision exp.  The normaliser Q' is summed over the
 * replicas in a fixed two-level tree (32 lanes inside each chunk of 256
 * slots, then 32 lanes over the chunk sums), and each replica has its own
 * Poisson mean.
 * Everything else (random keys, Poisson walk, slot order, checkerboard
 * order) is as for the +-1 oracle in pa_oracle.c.
 */
#include "pa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OG_SCALE_BITS 15
#define OG_INV_SCALE 0x1.0p-15

/* ------------------------------------------------------------------------
 * fexp: exp(x) for x <= 0 in single precision, the same on every IEEE
 * machine.  Cody & Waite reduction with a 16-bit head of ln2 (k * head exact
 * for |k| <= 151), degree-7 Taylor polynomial in Horner form with fused
 * multiply-adds (truncation below 2^-27 for |r| <= ln2/2), scaling by 2^k in
 * two factors below the normal range.  Coefficients c_0 = 1,
 * c_j = c_{j-1} / j rounded to single precision.
 *   head = floor(ln2 * 2^16) / 2^16, tail = ln2 - head (nearest float),
 *   1/ln2 to nearest float.
 * ---------------------------------------------------------------------- */
#define FEXP_INV_LN2 0x1.715476p+0f
#define FEXP_LN2_HI 0x1.62e4p-1f
#define FEXP_LN2_LO 0x1.7f7d1cp-20f
#define FEXP_SHIFT 0x1.8p23f
#define FEXP_DEGREE 7

static float fexp_coef[FEXP_DEGREE + 1];
static int fexp_ready = 0;

static void fexp_init(void) {
  if (fexp_ready) return;
  fexp_coef[0] = 1.0f;
  for (int j = 1; j <= FEXP_DEGREE; j++) fexp_coef[j] = fexp_coef[j - 1] / (float)j;
  fexp_ready = 1;
}

static float pow2f_i(int k) { /* 2^k, -126 <= k <= 127 */
  uint32_t bits = (uint32_t)(k + 127) << 23;
  float f;
  memcpy(&f, &bits, sizeof f);
  return f;
}

float og_fexp(float x) {
  fexp_init();
  if (x != x) return x;
  if (x > 0.0f) return NAN;
  if (x < -104.0f) return 0.0f;
  float t = x * FEXP_INV_LN2;
  float kf = (t + FEXP_SHIFT) - FEXP_SHIFT;
  float a = kf * FEXP_LN2_HI;
  float b = x - a;
  float c = kf * FEXP_LN2_LO;
  float r = b - c;
  float p = fexp_coef[FEXP_DEGREE];
  for (int j = FEXP_DEGREE - 1; j >= 0; j--) p = fmaf(p, r, fexp_coef[j]);
  int k = (int)kf;
  if (k >= -126) return p * pow2f_i(k);
  return (p * pow2f_i(k + 64)) * pow2f_i(-64);
}

/* Metropolis decision for a rise dE_q > 0 at inverse temperature beta with
 * uniform u (32 bits). */
int og_accept(double beta, int32_t dE_q, uint32_t u) {
  float bf = (float)beta;
  float ef = (float)dE_q;
  float x = -((bf * ef) * (float)OG_INV_SCALE);
  float p = og_fexp(x);
  float lim = p * 16777216.0f; /* p * 2^24 */
  float u24 = (float)(u >> 8);
  return u24 < lim;
}

/* ------------------------------------------------------------------------ */
static void philox_seeded_g(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                            uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  or_philox(ctr, key, out);
}

typedef struct {
  int64_t nb;
  int32_t J;
} og_edge;

struct og_run {
  int dim, Lx, Ly, Lz;
  int64_t N, Nb;
  int64_t* bond_i;
  int64_t* bond_j;
  int32_t* bond_J;
  int* deg;
  og_edge* adj;
  int8_t* colour;
  int64_t* lab_w;
  int* lab_p;
  int S; /* sites of one colour per packed word (keying) */
  uint64_t seed;
  int64_t R, R_cap;
  int8_t *spins, *spins_next;
  int64_t *E, *E_next;
  int32_t* copies;
  int64_t copies_n;
  double beta, mbF, lnQ_last, Qp_last;
  int64_t step, sweeps, sumE;
  double sumE2;
};
typedef struct og_run og_run;

static int64_t og_energy_of(const og_run* r, const int8_t* s) {
  int64_t E = 0;
  for (int64_t b = 0; b < r->Nb; b++)
    E += (int64_t)r->bond_J[b] * s[r->bond_i[b]] * s[r->bond_j[b]];
  return E;
}

int64_t og_energy(const og_run* r, const int8_t* s) { return og_energy_of(r, s); }

static int og_add_bond(og_run* r, int64_t i, int64_t j, int32_t J, int64_t* nb) {
  if (J == 0) return OR_OK;
  if (i == j || r->colour[i] == r->colour[j]) return OR_ERR_INVALID;
  if (r->deg[i] >= 6 || r->deg[j] >= 6) return OR_ERR_INVALID;
  r->bond_i[*nb] = i; r->bond_j[*nb] = j; r->bond_J[*nb] = J;
  (*nb)++;
  r->adj[i * 6 + r->deg[i]].nb = j; r->adj[i * 6 + r->deg[i]].J = J; r->deg[i]++;
  r->adj[j * 6 + r->deg[j]].nb = i; r->adj[j * 6 + r->deg[j]].J = J; r->deg[j]++;
  return OR_OK;
}

void og_destroy(og_run* r) {
  if (!r) return;
  free(r->bond_i); free(r->bond_j); free(r->bond_J); free(r->deg); free(r->adj);
  free(r->colour); free(r->lab_w); free(r->lab_p);
  free(r->spins); free(r->spins_next); free(r->E); free(r->E_next); free(r->copies);
  free(r);
}

static void og_sums(og_run* r) {
  r->sumE = 0;
  r->sumE2 = 0.0;
  for (int64_t s = 0; s < r->R; s++) {
    r->sumE += r->E[s];
    double e = (double)r->E[s] * OG_INV_SCALE;
    r->sumE2 += e * e;
  }
}

/* Lattice, labels and the beta = 0 population as for the +-1 oracle
 * (Sec. 2); couplings are int32 fixed point ([3][N] or [N]). */
int og_create(int dim, int Lx, int Ly, int Lz, unsigned periodic, const int32_t* J,
              int64_t R0, int64_t R_cap, uint64_t seed, og_run** out) {
  fexp_init();
  if (!out || !J) return OR_ERR_INVALID;
  *out = NULL;
  if (dim == 1) { Ly = 1; Lz = 1; }
  else if (dim != 3) return OR_ERR_INVALID;
  if (Lx < 2 || Ly < 1 || Lz < 1) return OR_ERR_INVALID;
  if (dim == 3 && (Lx % 2 != 0 || Lx > 32)) return OR_ERR_INVALID;
  if (R0 < 1 || R_cap < R0) return OR_ERR_INVALID;
  og_run* r = (og_run*)calloc(1, sizeof(og_run));
  if (!r) return OR_ERR_OOM;
  r->dim = dim; r->Lx = Lx; r->Ly = Ly; r->Lz = Lz;
  r->N = (int64_t)Lx * Ly * Lz;
  r->seed = seed;
  r->R = R0; r->R_cap = R_cap;
  int64_t N = r->N;
  r->bond_i = malloc(sizeof(int64_t) * 3 * N);
  r->bond_j = malloc(sizeof(int64_t) * 3 * N);
  r->bond_J = malloc(sizeof(int32_t) * 3 * N);
  r->deg = calloc(N, sizeof(int));
  r->adj = calloc(N * 6, sizeof(og_edge));
  r->colour = malloc(N);
  r->lab_w = malloc(sizeof(int64_t) * N);
  r->lab_p = malloc(sizeof(int) * N);
  r->spins = malloc((size_t)(R_cap * N));
  r->spins_next = malloc((size_t)(R_cap * N));
  r->E = malloc(sizeof(int64_t) * R_cap);
  r->E_next = malloc(sizeof(int64_t) * R_cap);
  r->copies = calloc(R_cap, sizeof(int32_t));
  if (!r->bond_i || !r->bond_j || !r->bond_J || !r->deg || !r->adj || !r->colour || !r->lab_w ||
      !r->lab_p || !r->spins || !r->spins_next || !r->E || !r->E_next || !r->copies) {
    og_destroy(r);
    return OR_ERR_OOM;
  }
  int64_t nb = 0;
  int st = OR_OK;
  if (dim == 1) {
    for (int64_t i = 0; i < N; i++) r->colour[i] = (int8_t)(i & 1);
    for (int64_t i = 0; i < N && st == OR_OK; i++) st = og_add_bond(r, i, (i + 1) % N, J[i], &nb);
    for (int64_t i = 0; i < N; i++) { r->lab_w[i] = i >> 5; r->lab_p[i] = (int)(i & 31); }
    r->S = 16;
  } else {
    int ext[3] = {Lx, Ly, Lz};
    for (int z = 0; z < Lz; z++)
      for (int y = 0; y < Ly; y++)
        for (int x = 0; x < Lx; x++)
          r->colour[x + (int64_t)Lx * (y + (int64_t)Ly * z)] = (int8_t)((x + y + z) & 1);
    for (int d = 0; d < 3 && st == OR_OK; d++)
      for (int z = 0; z < Lz && st == OR_OK; z++)
        for (int y = 0; y < Ly && st == OR_OK; y++)
          for (int x = 0; x < Lx && st == OR_OK; x++) {
            int c[3] = {x, y, z};
            if (c[d] == ext[d] - 1 && !((periodic >> d) & 1)) continue;
            int n[3] = {x, y, z};
            n[d] = (c[d] + 1) % ext[d];
            int64_t i = x + (int64_t)Lx * (y + (int64_t)Ly * z);
            int64_t j = n[0] + (int64_t)Lx * (n[1] + (int64_t)Ly * n[2]);
            st = og_add_bond(r, i, j, J[(int64_t)d * N + i], &nb);
          }
    int k = 1;
    for (int dd = Lz; dd >= 1; dd--)
      if (Lz % dd == 0 && dd * Lx <= 32) { k = dd; break; }
    int G = Lz / k;
    r->S = k * Lx / 2;
    for (int z = 0; z < Lz; z++)
      for (int y = 0; y < Ly; y++)
        for (int x = 0; x < Lx; x++) {
          int64_t i = x + (int64_t)Lx * (y + (int64_t)Ly * z);
          r->lab_w[i] = (int64_t)y * G + (z % G);
          r->lab_p[i] = (z / G) * Lx + x;
        }
  }
  if (st != OR_OK) { og_destroy(r); return st; }
  r->Nb = nb;
  for (int64_t s = 0; s < R0; s++) {
    int8_t* sig = r->spins + s * N;
    for (int64_t i = 0; i < N; i++) {
      uint32_t o[4];
      int64_t w = r->lab_w[i];
      philox_seeded_g(seed, (uint32_t)(w >> 2), (uint32_t)s, 0u, OR_TAG_INIT, o);
      sig[i] = ((o[w & 3] >> r->lab_p[i]) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
    r->E[s] = og_energy_of(r, sig);
  }
  r->mbF = (double)N * 0x1.62e42fefa39efp-1; /* ln Omega = N ln 2 */
  og_sums(r);
  *out = r;
  return OR_OK;
}

static uint32_t og_sweep_uniform(const og_run* r, int64_t i, int64_t s, uint32_t T, int c) {
  int64_t rank = r->lab_w[i] * r->S + (r->lab_p[i] >> 1);
  uint32_t o[4];
  philox_seeded_g(r->seed, (uint32_t)(rank >> 2), (uint32_t)s, T, OR_TAG_SWEEP + (uint32_t)c, o);
  return o[rank & 3];
}

/* theta checkerboard sweeps of one replica in slot s from global sweep T0;
 * returns the tracked energy change. */
static int64_t og_sweep_one(const og_run* r, int8_t* sig, int64_t s, int64_t T0, double beta, int theta) {
  int64_t dsum = 0;
  for (int t = 0; t < theta; t++) {
    uint32_t T = (uint32_t)(T0 + t);
    for (int c = 0; c < 2; c++)
      for (int64_t i = 0; i < r->N; i++) {
        if (r->colour[i] != c) continue;
        int32_t h = 0;
        for (int e = 0; e < r->deg[i]; e++) h += r->adj[i * 6 + e].J * sig[r->adj[i * 6 + e].nb];
        int32_t dE = -2 * sig[i] * h;
        int flip = dE <= 0 || og_accept(beta, dE, og_sweep_uniform(r, i, s, T, c));
        if (flip) {
          sig[i] = (int8_t)(-sig[i]);
          dsum += dE;
        }
      }
  }
  return dsum;
}

int og_sweep_replica(const og_run* r, int8_t* sigma, int64_t slot, int64_t T0, double beta, int theta,
                     int64_t* E_out) {
  int64_t E0 = og_energy_of(r, sigma);
  int64_t Et = E0 + og_sweep_one(r, sigma, slot, T0, beta, theta);
  int64_t Ere = og_energy_of(r, sigma);
  if (Et != Ere) return OR_ERR_STATE;
  if (E_out) *E_out = Ere;
  return OR_OK;
}

/* Q' by the fixed tree over replicas, ln Q, and the copy counts (Sec. 2,
 * Eqs. (1)-(2); Algorithm, resampling). */
static int og_resample_counts(const og_run* r, const int64_t* E, int64_t R, double dbeta, int64_t R_target,
                              int64_t step, int32_t* copies, int64_t* Rn_out, double* Qp_out,
                              double* lnQ_out) {
  int64_t Emin = E[0];
  for (int64_t j = 1; j < R; j++)
    if (E[j] < Emin) Emin = E[j];
  double* w = malloc(sizeof(double) * R);
  if (!w) return OR_ERR_OOM;
  for (int64_t j = 0; j < R; j++)
    w[j] = or_pexp(-(dbeta * ((double)(E[j] - Emin) * OG_INV_SCALE)));
  /* Two-level fixed tree.  Level 1, chunk c of 256 slots: lane l sums w_j,
   * j = 256c + l + 32i (i = 0..7, j < R) in increasing i, then butterfly
   * levels 16, 8, 4, 2, 1.  Level 2: lane l sums the chunk sums c = l, l+32,
   * ... in increasing c, then the same butterfly. */
  int64_t nch = (R + 255) / 256;
  double* chunk = malloc(sizeof(double) * nch);
  if (!chunk) { free(w); return OR_ERR_OOM; }
  double lane[32];
  for (int64_t cidx = 0; cidx < nch; cidx++) {
    int64_t base = 256 * cidx;
    for (int l = 0; l < 32; l++) {
      double acc = 0.0;
      for (int i = 0; i < 8; i++) {
        int64_t j = base + l + 32 * i;
        if (j < R) acc = acc + w[j];
      }
      lane[l] = acc;
    }
    for (int sh = 16; sh >= 1; sh >>= 1) {
      double nxt[32];
      for (int l = 0; l < 32; l++) nxt[l] = lane[l] + lane[l ^ sh];
      memcpy(lane, nxt, sizeof lane);
    }
    chunk[cidx] = lane[0];
  }
  for (int l = 0; l < 32; l++) {
    double acc = 0.0;
    for (int64_t cidx = l; cidx < nch; cidx += 32) acc = acc + chunk[cidx];
    lane[l] = acc;
  }
  for (int sh = 16; sh >= 1; sh >>= 1) {
    double nxt[32];
    for (int l = 0; l < 32; l++) nxt[l] = lane[l] + lane[l ^ sh];
    memcpy(lane, nxt, sizeof lane);
  }
  double Qp = lane[0];
  free(chunk);
  double lnQ = log(Qp) - log((double)R) - dbeta * ((double)Emin * OG_INV_SCALE);
  int64_t Rn = 0;
  for (int64_t j = 0; j < R; j++) {
    double a = ((double)R_target * w[j]) / Qp;
    int64_t m = 1;
    if (a > 32.0) m = (int64_t)ceil(a / 32.0);
    double am = a / (double)m;
    double p0 = or_pexp(-am);
    int64_t cj = 0;
    for (int64_t piece = 0; piece < m; piece++) {
      uint32_t o[4];
      philox_seeded_g(r->seed, (uint32_t)piece, (uint32_t)j, (uint32_t)step, OR_TAG_RESAMPLE, o);
      cj += or_poisson_piece(or_u53(o[0], o[1]), am, p0);
    }
    copies[j] = (int32_t)(cj > 0x7FFFFFFF ? 0x7FFFFFFF : cj);
    Rn += cj;
  }
  free(w);
  *Rn_out = Rn;
  *Qp_out = Qp;
  *lnQ_out = lnQ;
  return OR_OK;
}

int og_resample(const og_run* r, const int64_t* E, int64_t R, double beta, double beta_next, int64_t R_target,
                int64_t step, int32_t* copies, int64_t* Rn, double* Qp, double* lnQ) {
  if (!r || !E || !copies || R < 1 || !(beta_next >= beta)) return OR_ERR_INVALID;
  return og_resample_counts(r, E, R, beta_next - beta, R_target, step, copies, Rn, Qp, lnQ);
}

int og_step(og_run* r, double beta_next, int theta, int64_t R_target) {
  if (!r || theta < 0 || R_target < 1 || !(beta_next >= r->beta)) return OR_ERR_INVALID;
  double dbeta = beta_next - r->beta;
  int64_t N = r->N, R = r->R, Rn;
  double Qp, lnQ;
  int st = og_resample_counts(r, r->E, R, dbeta, R_target, r->step, r->copies, &Rn, &Qp, &lnQ);
  if (st != OR_OK) return st;
  r->copies_n = R;
  if (Rn == 0) return OR_ERR_EXTINCT;
  if (Rn > r->R_cap) return OR_ERR_CAPACITY;
  int64_t s = 0;
  for (int64_t j = 0; j < R; j++)
    for (int32_t q = 0; q < r->copies[j]; q++, s++) {
      memcpy(r->spins_next + s * N, r->spins + j * N, (size_t)N);
      r->E_next[s] = r->E[j];
    }
  for (int64_t q = 0; q < Rn; q++) {
    int8_t* sig = r->spins_next + q * N;
    int64_t Et = r->E_next[q] + og_sweep_one(r, sig, q, r->sweeps, beta_next, theta);
    int64_t Ere = og_energy_of(r, sig);
    if (Et != Ere) return OR_ERR_STATE;
    r->E_next[q] = Ere;
  }
  int8_t* tsp = r->spins; r->spins = r->spins_next; r->spins_next = tsp;
  int64_t* tE = r->E; r->E = r->E_next; r->E_next = tE;
  r->R = Rn;
  r->beta = beta_next;
  r->mbF = r->mbF + lnQ;
  r->lnQ_last = lnQ;
  r->Qp_last = Qp;
  r->step += 1;
  r->sweeps += theta;
  og_sums(r);
  return OR_OK;
}

int og_sweep_fixed(og_run* r, double beta, int theta) {
  for (int64_t s = 0; s < r->R; s++) {
    int8_t* sig = r->spins + s * r->N;
    int64_t Et = r->E[s] + og_sweep_one(r, sig, s, r->sweeps, beta, theta);
    int64_t Ere = og_energy_of(r, sig);
    if (Et != Ere) return OR_ERR_STATE;
    r->E[s] = Ere;
  }
  r->sweeps += theta;
  og_sums(r);
  return OR_OK;
}

int og_get_state(const og_run* r, or_state* o, double* sumE2) {
  o->beta = r->beta; o->R = r->R; o->minus_beta_F = r->mbF;
  o->lnQ_last = r->lnQ_last; o->Qprime_last = r->Qp_last;
  o->step = r->step; o->sweeps = r->sweeps;
  o->sumE = r->sumE; o->sumE2 = 0;
  o->N = r->N; o->Nb = r->Nb; o->R_cap = r->R_cap;
  if (sumE2) *sumE2 = r->sumE2;
  return OR_OK;
}

int64_t og_copy_spins(const og_run* r, int8_t* dst, int64_t max_replicas) {
  int64_t n = r->R < max_replicas ? r->R : max_replicas;
  memcpy(dst, r->spins, (size_t)(n * r->N));
  return n;
}

int64_t og_copy_energies(const og_run* r, int64_t* dst, int64_t max_replicas) {
  int64_t n = r->R < max_replicas ? r->R : max_replicas;
  memcpy(dst, r->E, sizeof(int64_t) * (size_t)n);
  return n;
}

int64_t og_copy_copies(const og_run* r, int32_t* dst, int64_t max_replicas) {
  int64_t n = r->copies_n < max_replicas ? r->copies_n : max_replicas;
  memcpy(dst, r->copies, sizeof(int32_t) * (size_t)n);
  return n;
}
