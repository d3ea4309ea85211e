/*
 * pa.h -- C ABI of the GB300 population-annealing library.
 *
 * Population annealing with weighted averages (J. Machta, "Population
 * annealing with weighted averages: a Monte Carlo method for rough free
 * energy landscapes", 2010) on Edwards-Anderson Ising spin glasses: couplings
 * J in {-1, 0, +1} on 3D periodic cubic lattices (even L, 2..16) and 1D
 * chains (open or periodic), Gaussian couplings (the paper's Sec. 4 model, on
 * a 2^-15 fixed-point grid) on 3D lattices (even L, 4..12) and chains, and
 * both models on general Lx x Ly x Lz boxes with open or periodic axes.
 *
 * Conventions shared by every entry point
 *  - Energy: E = sum over nearest-neighbour bonds of J_ij s_i s_j, the sign
 *    of the paper's Sec. 4 definition (J = +1 is antiferromagnetic).
 *  - 3D couplings: int8 array [3][N], N = L^3, site i = x + L (y + L z);
 *    J[d][i] couples site i to its +d neighbour (d = x, y, z) with periodic
 *    wrap.  Every entry must be -1 or +1.
 *  - 1D couplings: int8 array [N]; J[i] couples i and i+1, J[N-1] is the
 *    wrap bond (0 makes the chain open).  Entries in {-1, 0, +1}; an odd
 *    periodic chain is rejected (not bipartite); 2 <= N <= 4096 (longer
 *    chains: PA_ERR_UNSUPPORTED).
 *  - Gaussian couplings (the model the paper studies, Sec. 4): int32 array
 *    in the 3D layout above holding J_q, the coupling J = J_q 2^-15 on a
 *    fixed-point grid; energies of such runs are integers E_q in the same
 *    units (E = E_q 2^-15), so energy differences are exact and only the
 *    Metropolis acceptance exp(-beta dE) is rounded (binary32 arithmetic on
 *    24-bit uniforms).
 *  - Pointers named host_* or given as plain arrays in these signatures are
 *    host memory; pointers named *_dev are device memory of the run's GPU.
 *    The caller keeps ownership of everything it passes; inputs are copied.
 *  - Every call returns PA_OK or one of the PA_ERR_* codes below and sets a
 *    per-thread message readable with pa_last_error().  INVALID, OOM and
 *    UNSUPPORTED are detected on the host before any work is queued and leave
 *    the handle unchanged.  CAPACITY and EXTINCT are detected on the device
 *    during a step: the step is not committed (population, free energy and
 *    counters stay as after the last good step), the code is sticky, and it
 *    is returned by the next synchronising call (pa_sync, pa_observables,
 *    pa_free_energy, pa_trajectory, pa_copy_*).
 *  - Steps are asynchronous on the run's stream (pa_opts.stream, else the
 *    default stream); only the calls listed above synchronise.
 *  - A handle may be used from one host thread at a time.
 *  - Per-device set-up (the deterministic exp coefficients in constant
 *    memory, the device address of pa_bootstrap_noalloc's scratch array) is
 *    done once per device and kept for the life of the process: after a
 *    cudaDeviceReset of a device this library has used, the library must not
 *    be used on that device again in the same process.
 */
#ifndef PA_H
#define PA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PA_OK 0
#define PA_ERR_INVALID 1     /* bad argument, beta decreasing, non-bipartite lattice */
#define PA_ERR_OOM 2         /* device allocation refused */
#define PA_ERR_CAPACITY 3    /* resampled population would exceed R_cap */
#define PA_ERR_EXTINCT 4     /* resampled population is empty */
#define PA_ERR_TIMEOUT 5     /* a bounded device or host wait ran out */
#define PA_ERR_CUDA 6        /* CUDA runtime error */
#define PA_ERR_UNSUPPORTED 7 /* lattice shape without a compiled kernel */

typedef struct pa_run pa_run;
typedef struct pa_batch pa_batch;

/* Device allocator hooks (the Python binding routes them to PyTorch's
 * caching allocator).  alloc returns NULL to refuse. */
typedef void* (*pa_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*pa_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

typedef struct pa_opts {
  int64_t R_cap;       /* population capacity; 0 = R0 + 10 ceil(sqrt R0) + 64 */
  void* stream;        /* cudaStream_t for all work of the handle; NULL = default stream */
  pa_alloc_fn alloc;   /* NULL = cudaMallocAsync on the stream */
  pa_free_fn free;
  void* alloc_ctx;
  int32_t max_steps;   /* capacity of the per-step on-device record; 0 = 4096 */
  int32_t threads_per_block; /* sweep kernel block size: 32, 64, 128 or 256 for every lattice;
                                512 or 1024 too for Gaussian cubic lattices of L <= 8 (the
                                kernel with per-site threshold tables; 512 is their default); a
                                lattice class that does not support the size takes its default;
                                0 = library default */
  int32_t threads_per_replica; /* threads sweeping one replica: cubic lattices 1, 2, 4 or 8 for
                                  +-1 couplings, 1, 2 or 4 for Gaussian ones (ranges of whole rows;
                                  PA_ERR_INVALID where the rows do not split so); +-1 chains 1, 2,
                                  4 or 8 (ranges of ceil(words / P) words); Gaussian chains and
                                  general boxes 1; 0 = library default */
} pa_opts;

/* Observables after the last committed step (Sec. 2: measured after the
 * resampling and the sweeps, so no weight factors are needed). */
typedef struct pa_obs {
  double beta;          /* current inverse temperature */
  int64_t R;            /* population size R~ */
  double E_mean;        /* sum_j E_j / R~ */
  double E2_mean;       /* sum_j E_j^2 / R~ */
  double lnQ_last;      /* ln Q of the last step, Eq. (2) */
  double minus_beta_F;  /* -beta F~, Eq. (4) (ln Omega = N ln 2 included) */
  int64_t step;         /* annealing steps committed */
  int64_t sweeps;       /* Metropolis sweeps per replica so far */
  int64_t sumE;         /* exact integer sums over the population */
  int64_t sumE2;
} pa_obs;

/* Library version (major*10000 + minor*100 + patch). */
int pa_version(void);
/* Message of the last failing call on this host thread ("" if none). */
const char* pa_last_error(void);
/* Self-check of the exact division used by the Poisson inverse-CDF walk
 * (Sec. 2, resampling; no counterpart in the paper): on the current device,
 * n >= 0 seeded pairs (x, k), x from random bits (every exponent, zero,
 * subnormals, infinities, NaNs; half of them near the walk's range 2^-60..2^6),
 * 1 <= k <= 512, divided by the library's integer division and by the
 * hardware division; *mismatches = the number of pairs whose results differ
 * in any bit (0 when the two agree).  Synchronous; PA_ERR_INVALID for n < 0
 * or a NULL pointer. */
int pa_check_division(int64_t n, uint64_t seed, int64_t* mismatches);
/* Self-check of the deterministic exponentials (no counterpart in the
 * paper): on the current device, n >= 0 seeded points, x uniform in
 * [-745, 0] for the double-precision exp of the reweighting factors, Poisson
 * tables and thresholds, and in [-103, 0] for the single-precision exp of
 * the Gaussian acceptance; *max_ulp_double / *max_ulp_float = the largest
 * distance, in units in the last place, from CUDA's exp / expf at the same
 * points.  Synchronous; PA_ERR_INVALID for n < 0 or a NULL pointer. */
int pa_check_exp(int64_t n, uint64_t seed, int64_t* max_ulp_double, int64_t* max_ulp_float);
/* Self-check of the counter-based generator (no counterpart in the paper):
 * on the current device, n >= 0 seeded (seed, subsequence, offset) triples,
 * the first four words of cuRAND's Philox4_32_10 generator initialised with
 * them against the library's Philox4x32-10 of the same key and counter, in
 * both forms its kernels use (round keys bumped on the fly and precomputed);
 * *mismatches = the number of differing results (0 when all agree).
 * Synchronous; PA_ERR_INVALID for n < 0 or a NULL pointer, PA_ERR_CUDA if
 * the device refuses. */
int pa_check_philox(int64_t n, uint64_t seed, int64_t* mismatches);
/* The integer form of the Gaussian Metropolis decision (Sec. 4 couplings;
 * the check behind the kernels' threshold tables, no counterpart in the
 * paper): for n >= 0 fixed-point energy changes dE[i] (host array) at
 * inverse temperature beta >= 0, thr[i] (host array) = the threshold the
 * threshold-table sweep kernels compare with: a rise dE is accepted with
 * uniform u iff (u >> 8) < thr, which equals accepting iff
 * float(u >> 8) < float(fexp(-(float(beta) float(dE)) 2^-15) 2^24); 2^24 for
 * dE <= 0.  Computed on the current device; synchronous; PA_ERR_INVALID for
 * n < 0, beta < 0 or NULL arrays with n > 0. */
int pa_gauss_thresholds(double beta, int64_t n, const int32_t* dE, uint32_t* thr);

/* Sec. 2, first step of the Algorithm ("Initialize R0 replicas at beta=0"):
 * R0 replicas, each spin +-1 with probability 1/2 from the counter-based
 * generator keyed by seed; -beta F~ = ln Omega = N ln 2 (Eq. (4) at beta=0).
 * couplings: host int8, layout above (3D: [3][L^3]; 1D: [L]).  L: lattice
 * edge (3D) or chain length (1D).  dim: 1 or 3.  R0 >= 1.  On success *out
 * owns all device memory of the run; release it with pa_destroy. */
int pa_create(const int8_t* couplings, int L, int dim, int64_t R0, uint64_t seed,
              pa_run** out);
/* pa_create with options (capacity, stream, allocator); opts may be NULL. */
int pa_create_ex(const int8_t* couplings, int L, int dim, int64_t R0, uint64_t seed,
                 const pa_opts* opts, pa_run** out);
/* pa_create_ex for Gaussian couplings (Sec. 4: J_ij drawn from a Gaussian of
 * mean 0 and variance 1): couplings is a host int32 array of J_q (J = J_q
 * 2^-15), |J_q| <= 2^18 and sum |J_q| < 2^31 (else PA_ERR_INVALID).
 * dim 3: [3][L^3], L even in 4..12 (else PA_ERR_UNSUPPORTED).  dim 1: a
 * chain of L = N spins, [N] in the 1D layout (J_q[N-1] the wrap bond, 0 for
 * an open chain), 2 <= N <= 4096; the paper's 1D model is the periodic
 * chain.  The run takes every other call of this header that takes a
 * pa_run, with these differences: pa_observables gives E_mean and E2_mean in physical units,
 * sumE in units of 2^-15 and sumE2 = 0 (the exact sum of E_q^2 needs more
 * than 64 bits); pa_trajectory writes sumE in units of 2^-15 and zeros for
 * sumE2 (pa_trajectory_energy has both moments); pa_copy_energies gives E_q.
 * Q of Eq. (2) is summed over replicas (no energy histogram): w_j =
 * exp[-(beta'-beta)(E_j - E_min)] summed in a fixed two-level tree (chunks of
 * 256 replicas, 32 lanes each level), so Q and -beta F~ do not depend on
 * scheduling. */
int pa_create_gauss(const int32_t* couplings, int L, int dim, int64_t R0, uint64_t seed,
                    const pa_opts* opts, pa_run** out);
/* A run on a general lattice (Sec. 4 nearest-neighbour bonds; Sec. 2
 * initialisation as pa_create).  dim 3: an Ls[0] x Ls[1] x Ls[2] box, site
 * i = x + Lx (y + Ly z), couplings [3][N] as for the cubic lattice; axis d
 * is periodic if bit d of periodic_mask is set, else open (the couplings
 * stored for the wrap bonds of an open axis are ignored).  A coupling of 0
 * is an absent bond.  Lx must be even (<= 32), and a periodic axis of odd
 * length or of length 1 with a nonzero wrap coupling is rejected (not
 * bipartite); otherwise PA_ERR_INVALID.  The periodic cubic case with a
 * compiled kernel (even L, 2..16 for +-1, 4..12 Gaussian) runs the cubic
 * kernels; other boxes run a general kernel (table-driven neighbours) up to
 * 2048 sites whose tables and spins fit one block's shared memory (else
 * PA_ERR_UNSUPPORTED).  dim 1: a chain of Ls[0] spins, periodic if bit 0 of
 * periodic_mask is set, else open (J[N-1] ignored).  Everything else as
 * pa_create_ex. */
int pa_create_lattice(const int8_t* couplings, const int Ls[3], int dim, unsigned periodic_mask,
                      int64_t R0, uint64_t seed, const pa_opts* opts, pa_run** out);
/* pa_create_lattice with Gaussian couplings (int32 J_q as for
 * pa_create_gauss). */
int pa_create_lattice_gauss(const int32_t* couplings, const int Ls[3], int dim,
                            unsigned periodic_mask, int64_t R0, uint64_t seed,
                            const pa_opts* opts, pa_run** out);
void pa_destroy(pa_run* run);
/* Sec. 2, first step of the Algorithm, again on an existing run: a fresh
 * beta = 0 population of R0 replicas drawn with `seed`, keeping the
 * couplings and the device memory of the run (no allocation).  Asynchronous;
 * clears a sticky device error. */
int pa_reset(pa_run* run, uint64_t seed);
/* Checkpoint and resume (no counterpart in the paper; the counter-based
 * random streams make a run's state its population, energies, histogram,
 * counters and per-step record).  pa_checkpoint_bytes gives the size of the
 * current state; pa_checkpoint writes it into a host buffer (synchronises;
 * PA_ERR_INVALID if the buffer is too small, the run's sticky error if it
 * failed); pa_restore loads it into a run created with the same lattice,
 * couplings (checked by hash) and a capacity large enough, which then
 * continues exactly as the checkpointed run would have. */
int pa_checkpoint_bytes(pa_run* run, size_t* bytes);
int pa_checkpoint(pa_run* run, void* host_buf, size_t bytes);
int pa_restore(pa_run* run, const void* host_buf, size_t bytes);
/* Measurement hook (no counterpart in the paper).  enable = k >= 1 starts
 * timing every k-th sweep-kernel launch of the run (the first, the (k+1)-th,
 * ...; k = 1: all of them) with CUDA events on the run's stream and zeroes
 * the counters; enable = 0 synchronises, stops timing and writes the summed
 * milliseconds of the timed sweep launches, their number and the number of
 * kernels the run launched since timing was enabled.  Any output pointer may
 * be NULL; enable < 0 is PA_ERR_INVALID. */
int pa_kernel_time(pa_run* run, int enable, double* sweep_ms, int64_t* sweep_launches,
                   int64_t* kernel_launches);
/* Launch shape of the run's sweep kernel (no counterpart in the paper):
 * threads per block and threads per replica (see pa_opts).  Either output
 * may be NULL. */
int pa_sweep_shape(pa_run* run, int32_t* threads_per_block, int32_t* threads_per_replica);

/* One annealing step beta -> beta_next (Sec. 2 and its Algorithm, one pass
 * of the loop body): reweighting factors exp[-(beta'-beta) E_j], the
 * normaliser Q of Eq. (2) and -beta F~ += ln Q (Eqs. (3)-(4)), Poisson
 * copy counts with means (R/R~) tau_j of Eq. (1) and the population-size
 * target R = R0, the copy of the surviving replicas, then `sweeps`
 * checkerboard Metropolis sweeps at beta_next on every replica, then the
 * energy observables.  beta_next >= current beta (else PA_ERR_INVALID);
 * sweeps >= 0.  Asynchronous. */
int pa_step(pa_run* run, double beta_next, int sweeps);
/* pa_step with an explicit population target R_beta' (Sec. 4 varies it with
 * temperature: R = 1000 below beta = 0.9 and 3000 above).  R_target >= 1. */
int pa_step_target(pa_run* run, double beta_next, int sweeps, int64_t R_target);
/* The next n_steps steps of the Algorithm at once: step k goes to
 * betas[k] with thetas[k] sweeps (NULL: 10 each) and population target
 * R_targets[k] (NULL: R0), host arrays of n_steps entries, betas
 * non-decreasing from the run's current beta (else PA_ERR_INVALID before any
 * work is queued).  The schedule is copied to the device and the steps read
 * it there.  use_graph = 1 captures the n_steps steps once as a CUDA graph
 * and replays it (the graph is kept for later calls with the same n_steps,
 * e.g. after pa_reset); 0 launches step by step.  Asynchronous; results are
 * those of n_steps calls of pa_step_target.  At most max_steps steps per run
 * in all (pa_opts). */
int pa_run_schedule(pa_run* run, int n_steps, const double* betas, const int32_t* thetas,
                    const int64_t* R_targets, int use_graph);
/* Waits for the run's queued work; returns any sticky device error. */
int pa_sync(pa_run* run);
/* Observables of the current population (synchronises). */
int pa_observables(pa_run* run, pa_obs* out);
/* The dimensionless free-energy estimate -beta F~ of Eq. (4), i.e. ln Z~;
 * well defined at beta = 0 where it equals N ln 2 (synchronises). */
int pa_free_energy(pa_run* run, double* minus_beta_F);
/* Per-step record, index 0 = initial state, k = after step k (Sec. 2:
 * "ln Q is recorded" at each temperature).  Writes min(count, steps+1)
 * entries into each non-NULL host array; returns the count in *n. */
int pa_trajectory(pa_run* run, int64_t count, double* beta, double* lnQ,
                  double* minus_beta_F, int64_t* R, int64_t* sumE, int64_t* sumE2,
                  int64_t* n);
/* The energy moments of the same record in physical units, for either
 * coupling model: E_mean[k] = sum_j E_j / R~ and E2_mean[k] = sum_j E_j^2 / R~
 * after step k (Sec. 2: the energy is measured on the resampled, equilibrated
 * population).  Non-NULL host arrays get min(count, steps+1) entries; the
 * count goes to *n (synchronises). */
int pa_trajectory_energy(pa_run* run, int64_t count, double* E_mean, double* E2_mean, int64_t* n);

/* Sec. 4: overlap q = (1/N) sum_i s_i^(1) s_i^(2) between replica k of run a
 * and replica k of run b, k < min(R~_a, R~_b); *gamma = fraction with
 * |q| < qcut (Gamma = Prob(|q| < 0.2) for qcut = 0.2), *npairs the number of
 * pairs; hist_or_null (host, N+1 int64) receives counts of (N q + N)/2.
 * Both runs must share lattice geometry and GPU (synchronises both). */
int pa_overlap(pa_run* a, pa_run* b, double qcut, double* gamma, int64_t* npairs,
               int64_t* hist_or_null);

/* Sec. 3, Eqs. (5)-(6), with R^(r) e^{-beta F~_r} in place of
 * e^{-beta F~_r} when R_or_null is given (runs of different target size),
 * and Eq. (7): *mean = sum_r A_r w_r, *minus_beta_Fbar =
 * ln[(1/M) sum_r exp(-beta F~_r)].  Host arrays of length M >= 1; A may be
 * NULL (then *mean = 0).  Computed by a GPU kernel on device 0's default
 * stream (synchronises). */
int pa_weighted_average(int M, const double* minus_beta_F, const double* A,
                        const double* R_or_null, double* mean, double* minus_beta_Fbar);
/* Batched form on device memory: G groups of M runs each, arrays [G][M]
 * (A_dev and R_dev may be NULL), outputs [G].  Asynchronous on stream. */
int pa_weighted_average_dev(int G, int M, const double* x_dev, const double* A_dev,
                            const double* R_dev, double* mean_dev, double* fbar_dev,
                            void* stream);
/* Sec. 4, Eqs. (10) and (11): an observable of two independent runs (the
 * overlap probability Gamma) averaged over M pairs of runs with the pair
 * weights omega'_r = e^{-beta (F~_r^(1) + F~_r^(2))} / sum_r e^{...}, the
 * exponents given as minus_beta_F_1[r] = -beta F~_r^(1) and
 * minus_beta_F_2[r] = -beta F~_r^(2).  With R1_or_null and R2_or_null (both
 * or neither) each pair's weight carries the factor R^(1)_r R^(2)_r of runs
 * with different target sizes (Sec. 3).  *mean = sum_r A_r omega'_r (0 when A
 * is NULL); *minus_beta_Fbar2 = ln[(1/M) sum_r e^{x1_r + x2_r}], the Eq. (7)
 * estimate for the two-run system.  Host arrays of length M >= 1; R entries
 * must be positive (else PA_ERR_INVALID).  Computed by a GPU kernel on device
 * 0's default stream (synchronises). */
int pa_weighted_average_pairs(int M, const double* minus_beta_F_1, const double* minus_beta_F_2,
                              const double* A, const double* R1_or_null, const double* R2_or_null,
                              double* mean, double* minus_beta_Fbar2);
/* Batched form on device memory: G groups of M pairs, arrays [G][M] (A_dev,
 * R1_dev and R2_dev may be NULL; R1_dev and R2_dev both or neither), outputs
 * [G].  Asynchronous on stream. */
int pa_weighted_average_pairs_dev(int G, int M, const double* x1_dev, const double* x2_dev,
                                  const double* A_dev, const double* R1_dev, const double* R2_dev,
                                  double* mean_dev, double* fbar2_dev, void* stream);
/* Sec. 3 bootstrap: standard deviation (ddof 1) of the weighted mean and of
 * -beta F-bar over B resamples of size M drawn with the counter-based
 * generator keyed by seed.  Host arrays; R entries must be positive (else
 * PA_ERR_INVALID); synchronises. */
int pa_bootstrap(int M, const double* minus_beta_F, const double* A, const double* R_or_null,
                 int B, uint64_t seed, double* std_mean, double* std_minus_beta_F);

/* No counterpart in the paper.  pa_bootstrap without any device allocation,
 * for callers that cannot allocate: code that has given all device memory
 * to its own pool or to another framework, latency-critical loops that must
 * not pay for (or risk failing) an allocation mid-run, and deployments whose
 * device memory is fixed at start-up.  Inputs x_dev, A_dev (may be NULL),
 * R_dev (may be NULL) are device arrays of length M >= 1 on the current
 * device (the entries of R_dev must be positive: they are not read on the
 * host, and a zero or negative one gives NaN or infinite results); out_dev is a device array of 2 doubles receiving the standard
 * deviation (ddof 1) of the weighted mean and of -beta F-bar over B
 * resamples, 2 <= B <= PA_BOOTSTRAP_NOALLOC_MAX_B (else PA_ERR_INVALID,
 * nothing queued).  The per-resample scratch is one file-scope device array
 * of 2 * PA_BOOTSTRAP_NOALLOC_MAX_B doubles (64 KiB) that every GPU which
 * loads this library holds until the process exits.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * caches it; make that first call before any stream capture.  The call
 * makes no cudaMalloc, cudaFree or other allocating call, and each call
 * writes every scratch entry it reads, so nothing must be cleared between
 * calls; the array keeps the last call's values.  All calls share the one
 * array: calls that overlap on the GPU (different streams, no ordering)
 * race and give wrong results.  Asynchronous on `stream`; returns a PA_*
 * code without setting pa_last_error. */
#define PA_BOOTSTRAP_NOALLOC_MAX_B 4096
int pa_bootstrap_noalloc(int M, const double* x_dev, const double* A_dev, const double* R_dev,
                         int B, uint64_t seed, double* out_dev, void* stream);

/* Copies of the run's state for tests and analysis (synchronise):
 * spins as int8 +-1, [R][N] in natural site order; energies [R];
 * copy counts of the last step by old slot [R_prev].  Each writes
 * min(max_replicas, available) rows and returns the row count in *n. */
int pa_copy_spins(pa_run* run, int8_t* host_dst, int64_t max_replicas, int64_t* n);
int pa_copy_energies(pa_run* run, int32_t* host_dst, int64_t max_replicas, int64_t* n);
int pa_copy_copies(pa_run* run, int32_t* host_dst, int64_t max_replicas, int64_t* n);

/* ---- batched executor ----------------------------------------------------
 * Many independent runs (Sec. 3: "independent runs ... without communication
 * between processors") of mixed lattice sizes advanced together: every
 * kernel of a step covers all runs through a work table, and a whole
 * schedule is captured in one CUDA graph and launched once. */
typedef struct pa_run_spec {
  int32_t dim;              /* 1 or 3 */
  int32_t L;                /* edge (3D) or chain length (1D) */
  const int8_t* couplings;  /* host, layout as for pa_create */
  int64_t R0;
  uint64_t seed;
  int64_t R_cap;            /* 0 = default */
  /* Non-NULL: a Gaussian-coupling run (int32 J_q as for pa_create_gauss);
   * couplings is then ignored.  All runs of a batch share one model (else
   * PA_ERR_INVALID). */
  const int32_t* gauss_couplings;
  /* Ls[0] > 0 with dim = 3: a general box Ls[0] x Ls[1] x Ls[2] with the
   * periodic axes of periodic_mask, as for pa_create_lattice (L is then
   * ignored); Ls[0] = 0: the periodic cubic lattice of edge L. */
  int32_t Ls[3];
  uint32_t periodic_mask;
} pa_run_spec;

int pa_batch_create(int n_runs, const pa_run_spec* specs, const pa_opts* opts,
                    pa_batch** out);
void pa_batch_destroy(pa_batch* b);
/* Advance every run through n_steps annealing steps.  betas: host
 * [n_runs][n_steps] (per_run_schedule != 0) or [n_steps] shared; thetas and
 * R_targets likewise shaped or NULL (theta = 10, R_target = R0).
 * use_graph != 0 captures all steps in one CUDA graph and launches it once.
 * Asynchronous; pa_batch_sync waits and returns the first sticky error. */
int pa_batch_run(pa_batch* b, int n_steps, const double* betas, int per_run_schedule,
                 const int32_t* thetas, const int64_t* R_targets, int use_graph);
int pa_batch_sync(pa_batch* b, int32_t* host_errors_or_null);
/* Per-run records after the last step: host arrays [n_runs] (any may be NULL). */
int pa_batch_results(pa_batch* b, double* beta, double* minus_beta_F, int64_t* R,
                     int64_t* sumE, int64_t* sumE2, int64_t* step);
/* Per-run per-step records: host arrays [n_runs][count].  Gaussian runs:
 * sumE in units of 2^-15, zeros for sumE2 (in pa_batch_results too). */
int pa_batch_trajectory(pa_batch* b, int64_t count, double* minus_beta_F, int64_t* R,
                        int64_t* sumE, int64_t* sumE2);
/* pa_trajectory_energy for every run of a batch: host arrays
 * [n_runs][count] of the per-step energy moments in physical units. */
int pa_batch_energy(pa_batch* b, int64_t count, double* E_mean, double* E2_mean);
/* Sec. 3 estimators over independent runs, computed on the device from the
 * runs' own per-step records (no host copy of the records): the batch's runs
 * split into groups of M consecutive runs (n_runs divisible by M, else
 * PA_ERR_INVALID), and for every group g and record k < count (every run
 * must have count records, else PA_ERR_INVALID):
 *   E_bar[g][k]           = sum_r E_r omega_r, omega_r ∝ R^(r) e^{-beta F~_r}
 *                           (Eqs. (5)-(6) with the R factor; R^(r)
 *                           = the target population of the step, R0 at k = 0;
 *                           E_r = the run's mean energy, physical units);
 *   minus_beta_Fbar[g][k] = ln[(1/M) sum_r e^{-beta F~_r}] (Eq. (7));
 *   var_minus_beta_F[g][k]= Var over the group of -beta F~_r (ddof 1), the
 *                           paper's convergence diagnostic (Sec. 3).
 * Host arrays [n_runs / M][count], any may be NULL; synchronises; scratch
 * of 8 (3 M + 3) n_runs/M count bytes from the batch's allocator. */
int pa_batch_diagnostics(pa_batch* b, int M, int64_t count, double* E_bar,
                         double* minus_beta_Fbar, double* var_minus_beta_F);
/* Sec. 3 bootstrap errors of the two estimators of pa_batch_diagnostics, for
 * every group g of M consecutive runs and record k < count at once:
 * sd_E_bar[g][k] and sd_minus_beta_Fbar[g][k] are the sample standard
 * deviations (ddof 1) over B resamples of the group's M runs, resample b
 * drawing member floor(word0 M / 2^32) of Philox(key seed, ctr (b, i, 0,
 * TAG_BOOT)) for i < M (the draws of pa_bootstrap, the same for every group
 * and record).  Argument rules and errors as pa_batch_diagnostics, plus
 * 2 <= B <= 2^20; host arrays [n_runs / M][count], either may be NULL;
 * synchronises; scratch of 8 (3 M + 2 B + 2) n_runs/M count bytes from the
 * batch's allocator (PA_ERR_OOM if refused). */
int pa_batch_bootstrap(pa_batch* b, int M, int64_t count, int B, uint64_t seed,
                       double* sd_E_bar, double* sd_minus_beta_Fbar);
/* Sec. 4 overlap between runs of one batch, for n_pairs pairs at once:
 * gamma[p] = fraction of replicas k < min(R~_a, R~_b) with |q_k| < qcut,
 * q_k = (1/N) sum_i s_i s'_i for replica k of run run_a[p] and replica k of
 * run run_b[p] (the pairing of pa_overlap); npairs[p] (may be NULL) the
 * number of replica pairs.  Host arrays of n_pairs (1..65535) entries; the
 * runs of a pair must share the lattice (else PA_ERR_INVALID).  Computed in
 * one launch for all pairs; synchronises. */
int pa_batch_overlap(pa_batch* b, int n_pairs, const int32_t* run_a, const int32_t* run_b,
                     double qcut, double* gamma, int64_t* npairs);
/* Sec. 2, first step of the Algorithm, again for every run of a batch: fresh
 * beta = 0 populations of R0 replicas drawn with seeds[r] (NULL: each run's
 * current seed), keeping the couplings, the device memory and a captured
 * schedule graph (no allocation).  Asynchronous; clears sticky errors. */
int pa_batch_reset(pa_batch* b, const uint64_t* seeds);
/* Sec. 4, P(q): the histogram of the overlap for n_pairs pairs of runs of
 * one batch at once, the pairing of pa_batch_overlap: hist[p][i] = the
 * number of replicas k < min(R~_a, R~_b) of runs run_a[p], run_b[p] with
 * (N q_k + N) / 2 = i, i = 0 .. N.  Every run of every pair must have the
 * lattice of run_a[0] (else PA_ERR_INVALID); hist is a host array
 * [n_pairs][N + 1]; 1 <= n_pairs <= 65535; one launch for all pairs;
 * synchronises. */
int pa_batch_overlap_hist(pa_batch* b, int n_pairs, const int32_t* run_a, const int32_t* run_b,
                          int64_t* hist);
/* Sweep launch shape chosen for each lattice class by timing the
 * candidates on the batch's own populations at the current temperature (a
 * dry step of min(sweeps, 20) Metropolis sweeps, sweeps <= 0 meaning 10: pass
 * the schedule's sweeps per step, since a block's fixed cost weighs less the
 * more sweeps it runs; no state is committed): the block size, and for +-1 cubic
 * lattices the threads per replica (1, 2, 4 or 8 threads sweeping disjoint
 * ranges of whole rows; 1, 2 or 4 for Gaussian ones, whose candidates include
 * blocks of 512 and 1024 threads at L <= 8).  The bit packing of the lattice is not a candidate:
 * it is part of the random keying (a site's uniform is keyed by its word and
 * bit), so another packing would draw other random numbers.  Writes up to 8
 * (L, threads per block, threads per replica) triples (L < 0 for chains; any
 * array may be NULL); returns the count in *n. */
int pa_batch_autotune(pa_batch* b, int32_t sweeps, int32_t* host_L, int32_t* host_threads, int32_t* host_split,
                      int* n);
/* Spins of run r as int8 +-1, [R][N] (synchronises). */
int pa_batch_copy_spins(pa_batch* b, int r, int8_t* host_dst, int64_t max_replicas,
                        int64_t* n);
/* Checkpoint and resume of a whole batch (no counterpart in the paper): a
 * small header, then every run's state in the pa_checkpoint format, in run
 * order.  pa_batch_checkpoint_bytes gives the size; pa_batch_checkpoint
 * writes it into a caller-owned host buffer (synchronises; PA_ERR_INVALID if
 * the buffer is too small, the first failed run's sticky error if any run
 * failed); pa_batch_restore loads it into a batch created from the same run
 * specs (same number of runs; per run the same lattice, model, couplings by
 * hash and a capacity large enough), which then continues exactly as the
 * checkpointed batch would have, schedules given from the checkpoint's step
 * on.  Every run is checked before any is loaded: a refused restore
 * (PA_ERR_INVALID) leaves the batch as it was. */
int pa_batch_checkpoint_bytes(pa_batch* b, size_t* bytes);
int pa_batch_checkpoint(pa_batch* b, void* host_buf, size_t bytes);
int pa_batch_restore(pa_batch* b, const void* host_buf, size_t bytes);

/* ---- serving -------------------------------------------------------------
 * Annealing runs submitted as requests and advanced with continuous batching
 * (independent runs, Sec. 3): each pa_server_tick admits queued requests in
 * arrival order while their device memory fits the budget and a run slot is
 * free, advances every admitted run by up to `steps` annealing steps in
 * shared launches, and retires finished runs, releasing their memory.  A run's
 * result does not depend on what it was batched with (same arithmetic and
 * random streams as pa_run). */
typedef struct pa_server pa_server;

typedef struct pa_request {
  int32_t dim;              /* 1 or 3 */
  int32_t L;                /* edge (3D) or chain length (1D) */
  const int8_t* couplings;  /* host, layout as for pa_create; copied at submit */
  int64_t R0;               /* initial population and target of every step */
  uint64_t seed;
  int32_t n_steps;          /* annealing steps */
  int32_t theta;            /* sweeps per step */
  const double* betas;      /* host [n_steps], beta after each step, non-decreasing from 0 */
} pa_request;

typedef struct pa_result {
  int32_t status;           /* 0 queued, 1 running, 2 done, 3 failed (error holds the PA code),
                               4 cancelled */
  int32_t error;
  int64_t steps;            /* steps committed */
  int64_t R;                /* final population size */
  double beta;              /* final beta */
  double minus_beta_F;      /* final -beta F~ (Eq. (4)) */
  double E_mean;            /* final mean energy */
  int64_t sumE, sumE2;
  double submit_s, admit_s, done_s;  /* pa_server_clock() times */
  int64_t device_bytes;     /* device memory the run held */
  int64_t flips;            /* attempted spin flips, sum over steps of R~_k N theta */
} pa_result;

/* opts: stream / allocator / max_steps (0 = 1024) / threads_per_block;
 * hbm_budget_bytes <= 0 means 80 % of the free device memory at creation;
 * max_runs = size of the device run table. */
int pa_server_create(const pa_opts* opts, double hbm_budget_bytes, int max_runs, pa_server** out);
void pa_server_destroy(pa_server* s);
/* Queue a request (inputs are copied); *id identifies it.  PA_ERR_OOM if the
 * run alone exceeds the budget. */
int pa_server_submit(pa_server* s, const pa_request* req, int64_t* id);
/* Admit, advance up to `steps` steps, retire (synchronises).  A request
 * whose memory the allocator refuses stays first in the queue and is tried
 * again on the next tick; one whose set-up fails is marked failed alone. */
int pa_server_tick(pa_server* s, int steps, int32_t* n_active, int32_t* n_queued, int32_t* n_finished);
/* Status and, once finished, the result of request id; traj (host, may be
 * NULL) receives up to `count` values of -beta F~ after steps 0, 1, .... */
int pa_server_result(pa_server* s, int64_t id, pa_result* out, double* traj, int64_t count);
/* Seconds since the server was created (clock of the result timestamps). */
double pa_server_clock(pa_server* s);
/* Cancel request id (no counterpart in the paper): a queued request leaves
 * the queue; a running one gives back its run slot and device memory at once
 * (call it between ticks); both then report status 4 with the steps done so
 * far.  Finished, failed or cancelled requests are left as they are.  The
 * other runs are not affected: their results stay bit for bit the same.
 * PA_ERR_INVALID for an unknown id. */
int pa_server_cancel(pa_server* s, int64_t id);
/* Device memory the admitted runs hold, the admission budget, and the runs
 * resident now (any output may be NULL). */
int pa_server_memory(pa_server* s, int64_t* used_bytes, int64_t* budget_bytes, int32_t* runs_resident);

#ifdef __cplusplus
}
#endif
#endif /* PA_H */
