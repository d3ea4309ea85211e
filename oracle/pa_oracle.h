/*
 * pa_oracle.h -- plain CPU oracle for population annealing with weighted
 * averages (Machta 2010), applied to Edwards-Anderson Ising spin glasses.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It is deliberately slow and literal:
 * int8 spins (+1/-1) in natural site order, one site at a time, every random
 * word recomputed from its counter.
 *
 * Every function cites the passage of the paper it follows (Sec. 2 "The
 * Algorithm", Eqs. (1)-(4); Sec. 3 Eqs. (5)-(7);
 * Sec. 4 energy definition and Eqs. (10)-(11)).  Where the paper is
 * silent (random-number keying, Poisson sampler, sweep order, population
 * cap) the oracle follows the written specification of the method's
 * numerics that both sides implement independently.
 */
#ifndef PA_ORACLE_H
#define PA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_OK = 0,
  OR_ERR_INVALID = 1,
  OR_ERR_OOM = 2,
  OR_ERR_CAPACITY = 3,
  OR_ERR_EXTINCT = 4,
  OR_ERR_STATE = 5
};

/* Counter tags (fourth counter word) separating the random streams. */
#define OR_TAG_INIT     0x1A000000u
#define OR_TAG_RESAMPLE 0x2B000000u
#define OR_TAG_SWEEP    0x3C000000u /* + colour (0 or 1) */
#define OR_TAG_BOOT     0x4D000000u

/* Longest Poisson inverse-CDF walk for one piece of mean <= 32. */
#define OR_POISSON_KMAX 512

typedef struct or_run or_run;

typedef struct {
  double beta;          /* current inverse temperature */
  int64_t R;            /* current population size R~ */
  double minus_beta_F;  /* -beta F~ (Eq. (4)), includes ln Omega = N ln 2 */
  double lnQ_last;      /* ln Q of the last annealing step (Eq. (2)) */
  double Qprime_last;   /* Q' = sum_b n_b w_b of the last step */
  int64_t step;         /* annealing steps done */
  int64_t sweeps;       /* Metropolis sweeps done (global sweep counter) */
  int64_t sumE;         /* sum over the population of E_j */
  int64_t sumE2;        /* sum over the population of E_j^2 */
  int64_t N;            /* spins per replica */
  int64_t Nb;           /* bonds with nonzero coupling */
  int64_t R_cap;
} or_state;

/* Philox4x32-10 block (Salmon et al., SC'11): out = philox(ctr, key). */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Deterministic exp for x <= 0 (Cody-Waite reduction, degree-13 Taylor). */
double or_pexp(double x);
/* Top 53 bits of (w0:w1) as a double in [0,1). */
double or_u53(uint32_t w0, uint32_t w1);
/* One Poisson inverse-CDF walk of mean am with P(0)=p0 at uniform u. */
int32_t or_poisson_piece(double u, double am, double p0);
/* Uint32 Metropolis threshold for an energy rise dE > 0 at inverse temperature beta. */
uint32_t or_threshold(double beta, int dE);
/* Packed-word label (w, p) of a site and S, the sites of one colour per
 * word: the keying spec (the colour-c rank of the site is w*S + p div 2). */
int or_site_label(const or_run* r, int64_t site, int64_t* w, int* p, int* S);

/* dim = 3: lattice Lx x Ly x Lz, J is [3][N] (J[d][i] joins i to its +d
 * neighbour; ignored where axis d is open and i is on the last layer).
 * dim = 1: chain of Lx sites, J is [N], J[N-1] the wrap bond (0 = open). */
int or_create(int dim, int Lx, int Ly, int Lz, unsigned periodic_mask,
              const int8_t* J, int64_t R0, int64_t R_cap, uint64_t seed,
              or_run** out);
void or_destroy(or_run* r);
int or_step(or_run* r, double beta_next, int theta, int64_t R_target);
int or_sweep_fixed(or_run* r, double beta, int theta);
/* Steps 1-3 of an annealing step on given energies (no state change):
 * Q', ln Q and copy counts [R] by old slot; `step` keys the stream. */
int or_resample(const or_run* r, const int32_t* E, int64_t R, double beta,
                double beta_next, int64_t R_target, int64_t step, int32_t* copies,
                int64_t* Rn, double* Qp, double* lnQ);
/* theta sweeps at beta of one replica sigma (int8 +-1, [N], updated in
 * place) occupying slot `slot`, starting at global sweep T0; *E_out gets its
 * energy afterwards. */
int or_sweep_replica(const or_run* r, int8_t* sigma, int64_t slot, int64_t T0,
                     double beta, int theta, int64_t* E_out);
int or_get_state(const or_run* r, or_state* out);
int64_t or_copy_spins(const or_run* r, int8_t* dst, int64_t max_replicas);
int64_t or_copy_energies(const or_run* r, int32_t* dst, int64_t max_replicas);
int64_t or_copy_copies(const or_run* r, int32_t* dst, int64_t max_replicas);
int64_t or_energy_of(const or_run* r, const int8_t* sigma);
int or_overlap(const or_run* a, const or_run* b, double qcut, double* gamma,
               int64_t* npairs, int64_t* hist_or_null);

/* Sec. 3: weighted average over M runs (Eqs. (5)-(6), with the
 * R^(r) factor of the same section when R is given) and the free energy of
 * Eq. (7). */
int or_weighted_average(int M, const double* minus_beta_F, const double* A,
                        const double* R_or_null, double* mean,
                        double* minus_beta_Fbar);
int or_weighted_average_pairs(int M, const double* x1, const double* x2, const double* A,
                              const double* R1, const double* R2, double* mean, double* fbar2);
/* Sec. 3 bootstrap: B resamples of size M, sample std (ddof 1). */
int or_bootstrap(int M, const double* minus_beta_F, const double* A,
                 const double* R_or_null, int B, uint64_t seed,
                 double* std_mean, double* std_mbF);
/* Sec. 3 diagnostic: sample variance (ddof 1) of -beta F~ over runs. */
double or_variance(int M, const double* x);

/* ---- Gaussian couplings (pa_oracle_gauss.c) ------------------------------
 * Couplings are int32 fixed point, physical J = J_q * 2^-15; energies are
 * int64 in the same units. */
typedef struct og_run og_run;
float og_fexp(float x);
int og_accept(double beta, int32_t dE_q, uint32_t u);
int og_create(int dim, int Lx, int Ly, int Lz, unsigned periodic_mask, const int32_t* J,
              int64_t R0, int64_t R_cap, uint64_t seed, og_run** out);
void og_destroy(og_run* r);
int og_step(og_run* r, double beta_next, int theta, int64_t R_target);
int og_sweep_fixed(og_run* r, double beta, int theta);
int og_get_state(const og_run* r, or_state* out, double* sumE2_physical);
int64_t og_copy_spins(const og_run* r, int8_t* dst, int64_t max_replicas);
int64_t og_copy_energies(const og_run* r, int64_t* dst, int64_t max_replicas);
int64_t og_copy_copies(const og_run* r, int32_t* dst, int64_t max_replicas);
int64_t og_energy(const og_run* r, const int8_t* sigma);
int og_resample(const og_run* r, const int64_t* E, int64_t R, double beta, double beta_next,
                int64_t R_target, int64_t step, int32_t* copies, int64_t* Rn, double* Qp,
                double* lnQ);
int og_sweep_replica(const og_run* r, int8_t* sigma, int64_t slot, int64_t T0, double beta,
                     int theta, int64_t* E_out);

#ifdef __cplusplus
}
#endif
#endif
