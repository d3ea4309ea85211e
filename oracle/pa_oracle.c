/*
 * pa_oracle.c -- plain, slow, single-threaded CPU oracle for population
 * annealing with weighted averages (Machta 2010) on Ising spin glasses.
 *
 * TEST INFRASTRUCTURE ONLY: it exists to check the CUDA path; the product
 * library never links, loads or calls it.  Built with -ffp-contract=off so
 * that every floating-point operation is rounded exactly as written.
 *
 * Spins are int8 sigma = +1/-1 stored per site in natural order
 * i = x + Lx*(y + Ly*z); every bond is walked explicitly.  The only place the
 * packed-word geometry of the fast path appears is the keying label of
 * or_site_label(), which is part of the written random-number specification
 * (the paper fixes no random-number generator; both sides implement the
 * specification independently).
 */
#include "pa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Multipliers and Weyl key increments are the
 * published constants of the algorithm.
 * ---------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
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

static void philox_seeded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                          uint32_t c3, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  or_philox(ctr, key, out);
}

double or_u53(uint32_t w0, uint32_t w1) {
  uint64_t v = (((uint64_t)w0 << 32) | (uint64_t)w1) >> 11;
  return (double)v * 0x1.0p-53;
}

/* ------------------------------------------------------------------------
 * pexp: exp(x) for x <= 0, rounded identically on every IEEE-754 machine.
 * Cody & Waite (1980) argument reduction x = k ln2 + r with ln2 split in a
 * 40-bit head (exact products k*LN2_HI for |k| < 2^13) and a tail; then the
 * Taylor polynomial of degree 13 in Horner form with fused multiply-adds
 * (truncation error below 2^-57 for |r| <= ln2/2); then scaling by 2^k.
 * Coefficients follow the recurrence c_0 = 1, c_j = c_{j-1} / j, each
 * division rounded to nearest.
 *   LN2_HI  = floor(ln2 * 2^40) / 2^40
 *   LN2_LO  = ln2 - LN2_HI rounded to nearest
 *   INV_LN2 = 1/ln2 rounded to nearest
 * ---------------------------------------------------------------------- */
#define PEXP_INV_LN2 0x1.71547652b82fep+0
#define PEXP_LN2_HI 0x1.62e42fefa2000p-1
#define PEXP_LN2_LO 0x1.9ef35793c7673p-41
#define PEXP_ROUND_SHIFT 0x1.8p52
#define PEXP_DEGREE 13

static double pexp_coef[PEXP_DEGREE + 1];
static int pexp_ready = 0;

static void pexp_init(void) {
  if (pexp_ready) return;
  pexp_coef[0] = 1.0;
  for (int j = 1; j <= PEXP_DEGREE; j++) pexp_coef[j] = pexp_coef[j - 1] / (double)j;
  pexp_ready = 1;
}

static double pow2i(int k) { /* 2^k for -1022 <= k <= 1023 */
  uint64_t bits = (uint64_t)(k + 1023) << 52;
  double d;
  memcpy(&d, &bits, sizeof d);
  return d;
}

double or_pexp(double x) {
  pexp_init();
  if (x != x) return x;
  if (x > 0.0) return NAN; /* outside the specified domain */
  if (x < -746.0) return 0.0;
  double t = x * PEXP_INV_LN2;
  double kd = (t + PEXP_ROUND_SHIFT) - PEXP_ROUND_SHIFT; /* nearest integer, ties to even */
  double a = kd * PEXP_LN2_HI;
  double b = x - a;
  double c = kd * PEXP_LN2_LO;
  double r = b - c;
  double p = pexp_coef[PEXP_DEGREE];
  for (int j = PEXP_DEGREE - 1; j >= 0; j--) p = fma(p, r, pexp_coef[j]);
  int k = (int)kd;
  if (k >= -1022) return p * pow2i(k);
  return (p * pow2i(k + 200)) * pow2i(-200);
}

uint32_t or_threshold(double beta, int dE) {
  double prob = or_pexp(-(beta * (double)dE));
  double scaled = prob * 4294967296.0;
  if (scaled >= 4294967296.0) return 0xFFFFFFFFu;
  return (uint32_t)scaled; /* floor of a non-negative value */
}

int32_t or_poisson_piece(double u, double am, double p0) {
  int32_t k = 0;
  double P = p0, C = p0;
  while (u >= C && k < OR_POISSON_KMAX) {
    k = k + 1;
    P = (P * am) / (double)k;
    C = C + P;
  }
  return k;
}

/* ------------------------------------------------------------------------
 * Lattice and run state
 * ---------------------------------------------------------------------- */
typedef struct {
  int64_t nb;     /* neighbour site */
  int8_t J;       /* coupling of this bond */
} or_edge;

struct or_run {
  int dim, Lx, Ly, Lz;
  unsigned periodic;
  int64_t N;
  int64_t Nb;           /* stored bonds with J != 0 */
  int64_t* bond_i;      /* [Nb] */
  int64_t* bond_j;
  int8_t* bond_J;
  int* deg;             /* [N] number of incident bonds */
  or_edge* adj;         /* [N][6] */
  int8_t* colour;       /* [N] */
  int64_t* lab_w;       /* [N] keying label: packed word */
  int* lab_p;           /* [N] keying label: bit position in the word */
  int S;                /* sites of one colour per packed word (keying) */
  uint64_t seed;
  int64_t R, R_cap;
  int8_t* spins;        /* [R_cap][N] */
  int8_t* spins_next;
  int32_t* E;           /* [R_cap] */
  int32_t* E_next;
  int32_t* copies;      /* [R_cap] copy counts of the last step, by old slot */
  int64_t copies_n;
  double beta, mbF, lnQ_last, Qp_last;
  int64_t step, sweeps, sumE, sumE2;
};

static int64_t site_index(const or_run* r, int x, int y, int z) {
  return (int64_t)x + (int64_t)r->Lx * ((int64_t)y + (int64_t)r->Ly * z);
}

/* Keying label of a site: the packed word w it belongs to and its bit
 * position p inside the word.  3D: lanes of Lx bits, k lanes per word with
 * k the largest divisor of Lz such that k*Lx <= 32, G = Lz/k words per
 * (y) row; site (x,y,z) -> w = y*G + z mod G, p = (z div G)*Lx + x.
 * 1D: w = i div 32, p = i mod 32.  S = sites of one colour per word
 * (k*Lx/2 in 3D, 16 in 1D): the colour-c sites of the lattice are ranked
 * r = w*S + p div 2. */
static void make_labels(or_run* r) {
  if (r->dim == 1) {
    for (int64_t i = 0; i < r->N; i++) {
      r->lab_w[i] = i >> 5;
      r->lab_p[i] = (int)(i & 31);
    }
    r->S = 16;
    return;
  }
  int k = 1;
  for (int d = r->Lz; d >= 1; d--) {
    if (r->Lz % d == 0 && d * r->Lx <= 32) { k = d; break; }
  }
  int G = r->Lz / k;
  r->S = k * r->Lx / 2;
  for (int z = 0; z < r->Lz; z++)
    for (int y = 0; y < r->Ly; y++)
      for (int x = 0; x < r->Lx; x++) {
        int64_t i = site_index(r, x, y, z);
        r->lab_w[i] = (int64_t)y * G + (z % G);
        r->lab_p[i] = (z / G) * r->Lx + x;
      }
}

int or_site_label(const or_run* r, int64_t site, int64_t* w, int* p, int* S) {
  if (!r || site < 0 || site >= r->N) return OR_ERR_INVALID;
  *w = r->lab_w[site];
  *p = r->lab_p[site];
  *S = r->S;
  return OR_OK;
}

static int add_bond(or_run* r, int64_t i, int64_t j, int8_t J, int64_t* nb) {
  if (J == 0) return OR_OK;
  if (J != 1 && J != -1) return OR_ERR_INVALID;
  if (i == j) return OR_ERR_INVALID;                  /* self-loop */
  if (r->colour[i] == r->colour[j]) return OR_ERR_INVALID; /* not bipartite */
  if (r->deg[i] >= 6 || r->deg[j] >= 6) return OR_ERR_INVALID;
  r->bond_i[*nb] = i; r->bond_j[*nb] = j; r->bond_J[*nb] = J;
  (*nb)++;
  r->adj[i * 6 + r->deg[i]].nb = j; r->adj[i * 6 + r->deg[i]].J = J; r->deg[i]++;
  r->adj[j * 6 + r->deg[j]].nb = i; r->adj[j * 6 + r->deg[j]].J = J; r->deg[j]++;
  return OR_OK;
}

/* Energy of one configuration, E = sum over bonds of J_ij sigma_i sigma_j,
 * the paper's Sec. 4 definition (no minus sign). */
int64_t or_energy_of(const or_run* r, const int8_t* s) {
  int64_t E = 0;
  for (int64_t b = 0; b < r->Nb; b++)
    E += (int64_t)r->bond_J[b] * s[r->bond_i[b]] * s[r->bond_j[b]];
  return E;
}

static void free_run(or_run* r) {
  if (!r) return;
  free(r->bond_i); free(r->bond_j); free(r->bond_J); free(r->deg); free(r->adj);
  free(r->colour); free(r->lab_w); free(r->lab_p);
  free(r->spins); free(r->spins_next); free(r->E); free(r->E_next); free(r->copies);
  free(r);
}

void or_destroy(or_run* r) { free_run(r); }

int or_create(int dim, int Lx, int Ly, int Lz, unsigned periodic_mask,
              const int8_t* J, int64_t R0, int64_t R_cap, uint64_t seed,
              or_run** out) {
  pexp_init();
  if (!out || !J) return OR_ERR_INVALID;
  *out = NULL;
  if (dim == 1) { Ly = 1; Lz = 1; }
  else if (dim != 3) return OR_ERR_INVALID;
  if (Lx < 2 || Ly < 1 || Lz < 1) return OR_ERR_INVALID;
  if (dim == 3 && (Lx % 2 != 0 || Lx > 32)) return OR_ERR_INVALID;
  if (R0 < 1 || R_cap < R0) return OR_ERR_INVALID;
  or_run* r = (or_run*)calloc(1, sizeof(or_run));
  if (!r) return OR_ERR_OOM;
  r->dim = dim; r->Lx = Lx; r->Ly = Ly; r->Lz = Lz;
  r->periodic = periodic_mask;
  r->N = (int64_t)Lx * Ly * Lz;
  r->seed = seed;
  r->R = R0; r->R_cap = R_cap;
  int64_t N = r->N;
  int64_t maxb = 3 * N;
  r->bond_i = malloc(sizeof(int64_t) * maxb);
  r->bond_j = malloc(sizeof(int64_t) * maxb);
  r->bond_J = malloc(maxb);
  r->deg = calloc(N, sizeof(int));
  r->adj = calloc(N * 6, sizeof(or_edge));
  r->colour = malloc(N);
  r->lab_w = malloc(sizeof(int64_t) * N);
  r->lab_p = malloc(sizeof(int) * N);
  r->spins = malloc((size_t)(R_cap * N));
  r->spins_next = malloc((size_t)(R_cap * N));
  r->E = malloc(sizeof(int32_t) * R_cap);
  r->E_next = malloc(sizeof(int32_t) * R_cap);
  r->copies = calloc(R_cap, sizeof(int32_t));
  if (!r->bond_i || !r->bond_j || !r->bond_J || !r->deg || !r->adj || !r->colour ||
      !r->lab_w || !r->lab_p || !r->spins || !r->spins_next || !r->E || !r->E_next ||
      !r->copies) { free_run(r); return OR_ERR_OOM; }

  /* Lattice: colours and bonds (Sec. 4, nearest-neighbour bonds). */
  int64_t nb = 0;
  int st = OR_OK;
  if (dim == 1) {
    for (int64_t i = 0; i < N; i++) r->colour[i] = (int8_t)(i & 1);
    for (int64_t i = 0; i < N && st == OR_OK; i++)
      st = add_bond(r, i, (i + 1) % N, J[i], &nb);
  } else {
    for (int z = 0; z < Lz; z++)
      for (int y = 0; y < Ly; y++)
        for (int x = 0; x < Lx; x++)
          r->colour[site_index(r, x, y, z)] = (int8_t)((x + y + z) & 1);
    int ext[3] = {Lx, Ly, Lz};
    for (int d = 0; d < 3 && st == OR_OK; d++) {
      int periodic = (periodic_mask >> d) & 1;
      for (int z = 0; z < Lz && st == OR_OK; z++)
        for (int y = 0; y < Ly && st == OR_OK; y++)
          for (int x = 0; x < Lx && st == OR_OK; x++) {
            int c[3] = {x, y, z};
            if (c[d] == ext[d] - 1 && !periodic) continue; /* open boundary */
            int n[3] = {x, y, z};
            n[d] = (c[d] + 1) % ext[d];
            int64_t i = site_index(r, x, y, z);
            int64_t j = site_index(r, n[0], n[1], n[2]);
            st = add_bond(r, i, j, J[(int64_t)d * N + i], &nb);
          }
    }
  }
  if (st != OR_OK) { free_run(r); return st; }
  r->Nb = nb;
  make_labels(r);

  /* Sec. 2: R0 replicas at beta = 0, each an independent uniformly random
   * microstate.  Spin bit of site (w, p) in slot s: bit p of word (w mod 4)
   * of Philox(ctr = (w div 4, s, 0, TAG_INIT)); a set bit means sigma = -1. */
  for (int64_t s = 0; s < R0; s++) {
    int8_t* sig = r->spins + s * N;
    for (int64_t i = 0; i < N; i++) {
      uint32_t o[4];
      int64_t w = r->lab_w[i];
      philox_seeded(seed, (uint32_t)(w >> 2), (uint32_t)s, 0u, OR_TAG_INIT, o);
      uint32_t bit = (o[w & 3] >> r->lab_p[i]) & 1u;
      sig[i] = bit ? (int8_t)-1 : (int8_t)1;
    }
    r->E[s] = (int32_t)or_energy_of(r, sig);
  }
  /* Eq. (4) at beta = 0: -beta F~ = ln Omega = N ln 2. */
  r->beta = 0.0;
  r->mbF = (double)N * 0x1.62e42fefa39efp-1; /* ln 2 rounded to nearest */
  r->lnQ_last = 0.0;
  r->Qp_last = 0.0;
  r->step = 0; r->sweeps = 0;
  r->sumE = 0; r->sumE2 = 0;
  for (int64_t s = 0; s < R0; s++) {
    r->sumE += r->E[s];
    r->sumE2 += (int64_t)r->E[s] * r->E[s];
  }
  *out = r;
  return OR_OK;
}

/* ------------------------------------------------------------------------
 * Metropolis sweeps (Sec. 2: "equilibrating MCMC process at the new
 * temperature"; Algorithm, "Equilibrate replica j for theta sweeps").
 * Checkerboard order: in each sweep all colour-0 sites, then all colour-1
 * sites.  Site i of colour c in slot s at global sweep T, of rank
 * r = w*S + p div 2 among the colour-c sites, uses random word (r mod 4) of
 * Philox(ctr = (r div 4, s, T, TAG_SWEEP + c)).
 * Flip iff dE <= 0 or u < threshold(beta, dE).
 * ---------------------------------------------------------------------- */
static uint32_t sweep_uniform(const or_run* r, int64_t i, int64_t s, uint32_t T, int c) {
  int64_t rank = r->lab_w[i] * r->S + (r->lab_p[i] >> 1);
  uint32_t o[4];
  philox_seeded(r->seed, (uint32_t)(rank >> 2), (uint32_t)s, T, OR_TAG_SWEEP + (uint32_t)c, o);
  return o[rank & 3];
}

static void make_thresholds(double beta, uint32_t thr[7]) {
  thr[0] = 0;
  for (int d = 1; d <= 6; d++) thr[d] = or_threshold(beta, 2 * d);
}

/* theta sweeps of one replica held in slot s, starting at global sweep T0;
 * returns the tracked energy change. */
static int64_t sweep_one(const or_run* r, int8_t* sig, int64_t s, int64_t T0,
                         const uint32_t thr[7], int theta) {
  int64_t dEsum = 0;
  for (int t = 0; t < theta; t++) {
    uint32_t T = (uint32_t)(T0 + t);
    for (int c = 0; c < 2; c++) {
      for (int64_t i = 0; i < r->N; i++) {
        if (r->colour[i] != c) continue;
        int h = 0;
        for (int e = 0; e < r->deg[i]; e++) {
          const or_edge* ed = &r->adj[i * 6 + e];
          h += ed->J * sig[ed->nb];
        }
        int dE = -2 * sig[i] * h;
        int flip = 0;
        if (dE <= 0) flip = 1;
        else if (sweep_uniform(r, i, s, T, c) < thr[dE / 2]) flip = 1;
        if (flip) {
          sig[i] = (int8_t)(-sig[i]);
          dEsum += dE;
        }
      }
    }
  }
  return dEsum;
}

static int sweep_population(or_run* r, int8_t* spins, int32_t* E, int64_t R,
                            double beta, int theta) {
  uint32_t thr[7];
  make_thresholds(beta, thr);
  int64_t N = r->N;
  for (int64_t s = 0; s < R; s++) {
    int8_t* sig = spins + s * N;
    int64_t Etrack = E[s] + sweep_one(r, sig, s, r->sweeps, thr, theta);
    int64_t Ere = or_energy_of(r, sig);
    if (Ere != Etrack) return OR_ERR_STATE; /* tracked energy must equal recomputed */
    E[s] = (int32_t)Ere;
  }
  return OR_OK;
}

int or_sweep_replica(const or_run* r, int8_t* sigma, int64_t slot, int64_t T0,
                     double beta, int theta, int64_t* E_out) {
  if (!r || !sigma || theta < 0) return OR_ERR_INVALID;
  uint32_t thr[7];
  make_thresholds(beta, thr);
  int64_t E0 = or_energy_of(r, sigma);
  int64_t Et = E0 + sweep_one(r, sigma, slot, T0, thr, theta);
  int64_t Ere = or_energy_of(r, sigma);
  if (Et != Ere) return OR_ERR_STATE;
  if (E_out) *E_out = Ere;
  return OR_OK;
}

int or_sweep_fixed(or_run* r, double beta, int theta) {
  if (!r || theta < 0 || !(beta >= 0.0)) return OR_ERR_INVALID;
  int st = sweep_population(r, r->spins, r->E, r->R, beta, theta);
  if (st != OR_OK) return st;
  r->sweeps += theta;
  r->sumE = 0; r->sumE2 = 0;
  for (int64_t s = 0; s < r->R; s++) {
    r->sumE += r->E[s];
    r->sumE2 += (int64_t)r->E[s] * r->E[s];
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------
 * One annealing step beta -> beta' (Sec. 2 and its Algorithm):
 *   1. reweighting factors exp[-(beta'-beta) E_j], factored through the
 *      energy histogram as w_b = pexp(-dbeta * (E_b - E_min));
 *   2. Q (Eq. (2)) as Q' / R~ * exp(-dbeta E_min), with
 *      Q' = sum_b n_b w_b summed over a fixed 32-lane tree;
 *      ln Q is added to -beta F~ (Eqs. (3)-(4));
 *   3. copies of replica j ~ Poisson((R_beta'/R~) tau_j) with tau_j of
 *      Eq. (1), i.e. mean a_j = R_target w_j / Q';
 *   4. theta Metropolis sweeps at beta' on every new replica;
 *   5. observables after the sweeps (E, E^2 sums).
 * ---------------------------------------------------------------------- */
/* Steps 1-3 for a population with energies E[0..R): Q', ln Q and the copy
 * counts, in old-slot order.  `step` is the annealing-step index that keys
 * the resampling stream. */
static int resample_counts(const or_run* r, const int32_t* E, int64_t R, double dbeta,
                           int64_t R_target, int64_t step, int32_t* copies,
                           int64_t* Rn_out, double* Qp_out, double* lnQ_out) {
  int64_t nbins = r->Nb + 1;

  /* Energy histogram, bin b = (E + Nb)/2. */
  int64_t* hist = calloc(nbins, sizeof(int64_t));
  if (!hist) return OR_ERR_OOM;
  for (int64_t j = 0; j < R; j++) hist[(E[j] + r->Nb) / 2]++;
  int64_t bmin = 0;
  while (hist[bmin] == 0) bmin++;
  int64_t Emin = 2 * bmin - r->Nb;

  /* Q' over the fixed tree: lane l sums the nonempty bins b = l, l+32, ...
   * in increasing order (product, then sum, each rounded), then five
   * butterfly levels v[l] += v[l xor s] for s = 16, 8, 4, 2, 1. */
  double lane[32];
  for (int l = 0; l < 32; l++) {
    double acc = 0.0;
    for (int64_t b = l; b < nbins; b += 32) {
      if (hist[b] == 0) continue;
      double w = or_pexp(-(dbeta * (double)(2 * (b - bmin))));
      double term = (double)hist[b] * w;
      acc = acc + term;
    }
    lane[l] = acc;
  }
  for (int sh = 16; sh >= 1; sh >>= 1) {
    double nxt[32];
    for (int l = 0; l < 32; l++) nxt[l] = lane[l] + lane[l ^ sh];
    memcpy(lane, nxt, sizeof lane);
  }
  double Qp = lane[0];
  free(hist);
  double lnQ = log(Qp) - log((double)R) - dbeta * (double)Emin;

  /* Poisson copy counts, in old-slot order. */
  int64_t Rn = 0;
  for (int64_t j = 0; j < R; j++) {
    double w = or_pexp(-(dbeta * (double)(E[j] - Emin)));
    double a = ((double)R_target * w) / Qp;
    int64_t m = 1;
    if (a > 32.0) m = (int64_t)ceil(a / 32.0);
    double am = a / (double)m;
    double p0 = or_pexp(-am);
    int64_t cj = 0;
    for (int64_t piece = 0; piece < m; piece++) {
      uint32_t o[4];
      philox_seeded(r->seed, (uint32_t)piece, (uint32_t)j, (uint32_t)step,
                    OR_TAG_RESAMPLE, o);
      cj += or_poisson_piece(or_u53(o[0], o[1]), am, p0);
    }
    copies[j] = (int32_t)(cj > 0x7FFFFFFF ? 0x7FFFFFFF : cj);
    Rn += cj;
  }
  *Rn_out = Rn;
  *Qp_out = Qp;
  *lnQ_out = lnQ;
  return OR_OK;
}

int or_resample(const or_run* r, const int32_t* E, int64_t R, double beta,
                double beta_next, int64_t R_target, int64_t step, int32_t* copies,
                int64_t* Rn, double* Qp, double* lnQ) {
  if (!r || !E || !copies || R < 1 || R_target < 1 || !(beta_next >= beta))
    return OR_ERR_INVALID;
  return resample_counts(r, E, R, beta_next - beta, R_target, step, copies, Rn, Qp, lnQ);
}

int or_step(or_run* r, double beta_next, int theta, int64_t R_target) {
  if (!r || theta < 0 || R_target < 1) return OR_ERR_INVALID;
  if (!(beta_next >= r->beta)) return OR_ERR_INVALID;
  double dbeta = beta_next - r->beta;
  int64_t N = r->N, R = r->R;
  int64_t Rn;
  double Qp, lnQ;
  int rst = resample_counts(r, r->E, R, dbeta, R_target, r->step, r->copies, &Rn, &Qp, &lnQ);
  if (rst != OR_OK) return rst;
  r->copies_n = R;
  if (Rn == 0) return OR_ERR_EXTINCT;
  if (Rn > r->R_cap) return OR_ERR_CAPACITY;

  /* New population: copies of old slot j occupy consecutive new slots, in
   * increasing j. */
  int64_t s = 0;
  for (int64_t j = 0; j < R; j++) {
    for (int32_t q = 0; q < r->copies[j]; q++, s++) {
      memcpy(r->spins_next + s * N, r->spins + j * N, (size_t)N);
      r->E_next[s] = r->E[j];
    }
  }

  int st = sweep_population(r, r->spins_next, r->E_next, Rn, beta_next, theta);
  if (st != OR_OK) return st;

  int8_t* tsp = r->spins; r->spins = r->spins_next; r->spins_next = tsp;
  int32_t* tE = r->E; r->E = r->E_next; r->E_next = tE;
  r->R = Rn;
  r->beta = beta_next;
  r->mbF = r->mbF + lnQ;
  r->lnQ_last = lnQ;
  r->Qp_last = Qp;
  r->step += 1;
  r->sweeps += theta;
  r->sumE = 0; r->sumE2 = 0;
  for (int64_t q = 0; q < Rn; q++) {
    r->sumE += r->E[q];
    r->sumE2 += (int64_t)r->E[q] * r->E[q];
  }
  return OR_OK;
}

int or_get_state(const or_run* r, or_state* o) {
  if (!r || !o) return OR_ERR_INVALID;
  o->beta = r->beta; o->R = r->R; o->minus_beta_F = r->mbF;
  o->lnQ_last = r->lnQ_last; o->Qprime_last = r->Qp_last;
  o->step = r->step; o->sweeps = r->sweeps;
  o->sumE = r->sumE; o->sumE2 = r->sumE2;
  o->N = r->N; o->Nb = r->Nb; o->R_cap = r->R_cap;
  return OR_OK;
}

int64_t or_copy_spins(const or_run* r, int8_t* dst, int64_t max_replicas) {
  int64_t n = r->R < max_replicas ? r->R : max_replicas;
  memcpy(dst, r->spins, (size_t)(n * r->N));
  return n;
}

int64_t or_copy_energies(const or_run* r, int32_t* dst, int64_t max_replicas) {
  int64_t n = r->R < max_replicas ? r->R : max_replicas;
  memcpy(dst, r->E, sizeof(int32_t) * (size_t)n);
  return n;
}

int64_t or_copy_copies(const or_run* r, int32_t* dst, int64_t max_replicas) {
  int64_t n = r->copies_n < max_replicas ? r->copies_n : max_replicas;
  memcpy(dst, r->copies, sizeof(int32_t) * (size_t)n);
  return n;
}

/* Sec. 4: overlap q = (1/N) sum_i sigma_i^(1) sigma_i^(2) between replicas
 * of two independent runs, paired slot i with slot i; Gamma = Prob(|q| <
 * qcut), with |q| < qcut decided as |dot| < qcut * N in double. */
int or_overlap(const or_run* a, const or_run* b, double qcut, double* gamma,
               int64_t* npairs, int64_t* hist) {
  if (!a || !b || a->N != b->N) return OR_ERR_INVALID;
  int64_t n = a->R < b->R ? a->R : b->R;
  int64_t N = a->N, count = 0;
  if (hist) memset(hist, 0, sizeof(int64_t) * (size_t)(N + 1));
  for (int64_t i = 0; i < n; i++) {
    int64_t dot = 0;
    for (int64_t k = 0; k < N; k++) dot += a->spins[i * N + k] * b->spins[i * N + k];
    if (fabs((double)dot) < qcut * (double)N) count++;
    if (hist) hist[(dot + N) / 2]++;
  }
  *npairs = n;
  *gamma = n > 0 ? (double)count / (double)n : 0.0;
  return OR_OK;
}

/* ------------------------------------------------------------------------
 * Sec. 3: weighted averages over M independent runs.
 * omega_r = R_r e^{x_r} / sum_s R_s e^{x_s} (Eq. (6) with the R^(r) factor),
 * A-bar = sum_r A_r omega_r (Eq. (5)), evaluated with the largest
 * exponent factored out.  -beta F-bar = ln[(1/M) sum_r e^{x_r}] (Eq. (7),
 * last line).
 * ---------------------------------------------------------------------- */
int or_weighted_average(int M, const double* x, const double* A,
                        const double* Rw, double* mean, double* mbFbar) {
  if (M < 1 || !x) return OR_ERR_INVALID;
  double mu = -INFINITY, mux = -INFINITY;
  for (int r = 0; r < M; r++) {
    double y = x[r] + (Rw ? log(Rw[r]) : 0.0);
    if (y > mu) mu = y;
    if (x[r] > mux) mux = x[r];
  }
  double S = 0.0, SA = 0.0, Sx = 0.0;
  for (int r = 0; r < M; r++) {
    double y = x[r] + (Rw ? log(Rw[r]) : 0.0);
    double e = exp(y - mu);
    S = S + e;
    if (A) SA = SA + e * A[r];
    Sx = Sx + exp(x[r] - mux);
  }
  if (mean) *mean = A ? SA / S : 0.0;
  if (mbFbar) *mbFbar = mux + log(Sx) - log((double)M);
  return OR_OK;
}

/* Sec. 4, Eqs. (10)-(11): M pairs of independent runs, pair r weighted by
 * e^{-beta(F~_r^(1) + F~_r^(2))} = e^{x1_r + x2_r}, times R1_r R2_r when the
 * population factors of Sec. 3 are given; mean = sum_r A_r w_r / sum_r w_r and
 * fbar2 = ln[(1/M) sum_r e^{x1_r + x2_r}] (Eq. (7) for the two-run system).
 * Written as the sums of the definition, sequentially in r, with the largest
 * exponent factored out. */
int or_weighted_average_pairs(int M, const double* x1, const double* x2, const double* A,
                              const double* R1, const double* R2, double* mean, double* fbar2) {
  if (M < 1 || !x1 || !x2 || (R1 == NULL) != (R2 == NULL)) return OR_ERR_INVALID;
  double mu = -INFINITY, mux = -INFINITY;
  for (int r = 0; r < M; r++) {
    double x = x1[r] + x2[r];
    double y = x;
    if (R1) y = y + log(R1[r]) + log(R2[r]);
    if (y > mu) mu = y;
    if (x > mux) mux = x;
  }
  double S = 0.0, SA = 0.0, Sx = 0.0;
  for (int r = 0; r < M; r++) {
    double x = x1[r] + x2[r];
    double y = x;
    if (R1) y = y + log(R1[r]) + log(R2[r]);
    double e = exp(y - mu);
    S = S + e;
    if (A) SA = SA + e * A[r];
    Sx = Sx + exp(x - mux);
  }
  if (mean) *mean = A ? SA / S : 0.0;
  if (fbar2) *fbar2 = mux + log(Sx) - log((double)M);
  return OR_OK;
}

double or_variance(int M, const double* x) {
  if (M < 2) return 0.0;
  double m = 0.0;
  for (int r = 0; r < M; r++) m += x[r];
  m /= M;
  double v = 0.0;
  for (int r = 0; r < M; r++) v += (x[r] - m) * (x[r] - m);
  return v / (M - 1);
}

/* Bootstrap (Sec. 3): resample b draws index i of M as
 * floor(word0 * M / 2^32) of Philox(ctr = (b, i, 0, TAG_BOOT), key = seed). */
int or_bootstrap(int M, const double* x, const double* A, const double* Rw,
                 int B, uint64_t seed, double* std_mean, double* std_mbF) {
  if (M < 1 || B < 2 || !x) return OR_ERR_INVALID;
  double* xs = malloc(sizeof(double) * M);
  double* As = malloc(sizeof(double) * M);
  double* Rs = malloc(sizeof(double) * M);
  double* bm = malloc(sizeof(double) * B);
  double* bf = malloc(sizeof(double) * B);
  if (!xs || !As || !Rs || !bm || !bf) {
    free(xs); free(As); free(Rs); free(bm); free(bf);
    return OR_ERR_OOM;
  }
  for (int b = 0; b < B; b++) {
    for (int i = 0; i < M; i++) {
      uint32_t o[4];
      philox_seeded(seed, (uint32_t)b, (uint32_t)i, 0u, OR_TAG_BOOT, o);
      int k = (int)(((uint64_t)o[0] * (uint64_t)M) >> 32);
      xs[i] = x[k];
      As[i] = A ? A[k] : 0.0;
      Rs[i] = Rw ? Rw[k] : 1.0;
    }
    or_weighted_average(M, xs, A ? As : NULL, Rw ? Rs : NULL, &bm[b], &bf[b]);
  }
  *std_mean = sqrt(or_variance(B, bm));
  *std_mbF = sqrt(or_variance(B, bf));
  free(xs); free(As); free(Rs); free(bm); free(bf);
  return OR_OK;
}
