// pa_internal.h -- state shared by the host engine and the CUDA kernels.
//
// One RunDev per annealing run lives in device memory; every step kernel
// reads and writes it there, so a whole schedule runs without host round
// trips (and can be captured in one CUDA graph).
#pragma once
#include <stdint.h>

namespace pa {

// Counter tags (fourth counter word) separating the random streams.
constexpr uint32_t TAG_INIT = 0x1A000000u;
constexpr uint32_t TAG_RESAMPLE = 0x2B000000u;
constexpr uint32_t TAG_SWEEP = 0x3C000000u;  // + colour
constexpr uint32_t TAG_BOOT = 0x4D000000u;

constexpr int POISSON_KMAX = 512;  // longest inverse-CDF walk of one piece (mean <= 32)
constexpr int POISSON_TAB = 8;     // tabulated inverse-CDF steps per energy bin (+-1 couplings)
constexpr int CHUNK = 256;         // slots per block in the resampling kernels

// Error codes (mirrors pa.h).
constexpr int OK = 0, ERR_INVALID = 1, ERR_OOM = 2, ERR_CAPACITY = 3, ERR_EXTINCT = 4,
              ERR_TIMEOUT = 5, ERR_CUDA = 6, ERR_UNSUPPORTED = 7;

struct RunDev {
  // ---- static description
  uint64_t seed;
  int32_t dim;      // 1 or 3
  int32_t L;        // edge (3D) or chain length (1D)
  int32_t N;        // spins per replica
  int32_t Nb;       // bonds with nonzero coupling
  int32_t nbins;    // Nb + 1 energy bins, bin = (E + Nb) / 2
  int32_t W;        // packed 32-bit words per replica (multiple of 4)
  int32_t Wr;       // words actually used
  int64_t R_cap;
  int32_t max_steps;
  int32_t n_chunks;  // ceil(R_cap / CHUNK)
  uint32_t one;      // the constant 1, read at run time (keeps multiply-add compares opaque to the compiler)
  int32_t n_sched;   // valid entries of the device schedule; a run whose step reaches it is finished
  int32_t model;     // 0: couplings +-1 (or 0 in 1D); 1: Gaussian couplings, fixed point 2^-15
  int32_t gC0;       // sum of all couplings (Gaussian model: fixed point; general boxes: both models)
  // General Lx x Ly x Lz boxes (bx > 0; 0 for cubic lattices and chains):
  // extents, lanes per word (k), colour-c sites per word and the mask of the
  // used bits of a word.
  int32_t bx, by, bz, bk;
  int32_t bsites;
  uint32_t bvalid;

  // ---- device buffers
  uint32_t* spins[2];  // [R_cap][W] packed spins (bit set = spin -1)
  int32_t* E[2];       // [R_cap]
  uint32_t* hist[2];   // [nbins]
  uint32_t* bonds;     // coupling masks, see the sweep kernels
  int32_t* copies;     // [R_cap] copy counts by old slot
  int32_t* src;        // [R_cap] old slot of each new slot
  int64_t* chunk_sum;  // [n_chunks]
  int64_t* chunk_off;  // [n_chunks]
  int32_t* occ;        // [nbins] occupied bins of the step (unordered)
  double* bin_w;       // [nbins] reweighting factor of the step
  double* bin_am;      // [nbins] Poisson mean of one piece
  double* bin_p0;      // [nbins] exp(-bin_am)
  int64_t* bin_m;      // [nbins] number of pieces
  uint64_t* bin_thr;   // [nbins][POISSON_TAB] ceil(C_k 2^53), C_k the k-th partial sum of the walk
  double* bin_end;     // [nbins][2] P and C after the last tabulated step
  double* sched_beta;  // [max_steps] schedule for captured multi-step execution
  int32_t* sched_theta;
  int64_t* sched_R;
  int32_t* gJ;         // per-site couplings [2][6][Wr][S] (colour, direction, word, rank; Gaussian
                       // cubic lattices and general boxes), or J[N] (Gaussian chains)
  int32_t* gS;         // per-site coupling sums [2][Wr][S]
  int32_t* box_code;   // general boxes: [2][7][Wr][S] bit positions 32 w + p of the site (k = 0) and
                       // of its six neighbours (k = 1..6; the site itself where the bond is absent)
  double* w_rep;       // Gaussian model: [R_cap] reweighting factor of each replica
  double* chunk_q;     // Gaussian model: [n_chunks] Q' partial sums
  double* rec_beta;    // [max_steps + 1] per-step record
  double* rec_lnQ;
  double* rec_mbF;
  int64_t* rec_R;
  int64_t* rec_sumE;
  int64_t* rec_sumE2;

  // ---- dynamic state (device-owned)
  int32_t cur;         // buffer holding the population
  int32_t error;       // sticky PA error code
  int32_t skip;        // current step will not be committed
  int32_t theta_next;
  int32_t bmin;        // first occupied bin of hist[cur]
  int32_t pad0;
  int64_t R;           // population size R~
  int64_t R_next;
  int64_t Rt_next;     // target population of the step
  int64_t step;        // steps committed
  int64_t sweeps;      // sweeps per replica so far (global sweep counter)
  double beta, beta_next;
  double mbF, mbF_staged;
  double lnQ_last, lnQ_staged;
  double Qp_last, Qp_staged;
  int64_t sumE, sumE2;
  unsigned long long sumE_next, sumE2_next;  // two's-complement accumulators
  uint32_t thr[8];     // Metropolis thresholds at beta_next, index dE/2
  long long emin, emin_next;   // Gaussian model: lowest energy of the population
  // Gaussian model: sum of E_q^2 (E_q the fixed-point energy) accumulated
  // exactly as sumE2_next (low 32 bits of each E_q^2) + 2^32 sumE2hi_next
  // (high bits); sumE2d = that sum * 2^-30, i.e. the physical sum of E^2,
  // rounded once at commit.
  unsigned long long sumE2hi_next;
  double sumE2d;
};

// One block of a kernel covering runs: the run and its first slot.
struct Work {
  int32_t run;
  int32_t first;
};

}  // namespace pa
