// pa_step_kernels.cu -- the resampling half of an annealing step and the
// per-run bookkeeping (Sec. 2 and its Algorithm), plus set-up, read-out,
// overlap (Sec. 4) and weighted-average (Sec. 3) kernels.
//
// Step pipeline for a set of runs (all state on the device):
//   k_prepare  one warp per run: energy histogram -> Q' over the fixed
//              32-lane tree, ln Q and the staged -beta F~ (Eqs. (2), (4)),
//              per-bin Poisson means (Eq. (1)), Metropolis thresholds.
//   k_copies   one thread per replica: Poisson copy count (inverse CDF,
//              means above 32 split into pieces), per-chunk sums.
//   k_scan     one block per run: exclusive scan of the chunk sums, R~',
//              capacity / extinction check.
//   k_scatter  one thread per replica: source slot of every new slot.
//   k_sweep*   fused copy + sweeps + measurement (pa_sweep*.cu).
//   k_commit   one thread per run: commit the step or leave it untouched.
#include <math.h>

#include "pa_dexp.cuh"
#include "pa_divk.cuh"
#include "pa_gauss.cuh"

#include <algorithm>

namespace pa {

constexpr double LN2_NEAREST = 0x1.62e42fefa39efp-1;

// ceil(C 2^53) for 0 <= C < 2^10, from the bits of C (C = M 2^(e - 1075),
// M the 53-bit significand, so C 2^53 = M 2^(e - 1022)): the smallest
// integer U with U 2^-53 >= C.
__device__ __forceinline__ uint64_t cdf_threshold(double C) {
  const uint64_t bits = (uint64_t)__double_as_longlong(C);
  const int e = (int)(bits >> 52);
  if (e == 0) return bits != 0u ? 1u : 0u;  // zero, or below 2^-1022: C 2^53 < 1
  const uint64_t M = (bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int s = e - 1022;
  if (s >= 0) return M << s;
  if (s <= -64) return 1u;
  return (M + (1ull << -s) - 1u) >> -s;
}

// ---------------------------------------------------------------------------
// Set-up
// ---------------------------------------------------------------------------

// Coupling masks of a 3D cubic lattice from int8 J[3][N] (site i = x + L(y + L z)).
__global__ void k_setup_bonds3d(const int8_t* __restrict__ J, int L, int K, int G, int W,
                                uint32_t* __restrict__ bonds) {
  const int WR = L * G;
  const int N = L * L * L;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += gridDim.x * blockDim.x) {
    uint32_t m[6] = {0, 0, 0, 0, 0, 0};
    if (w < WR) {
      const int y = w / G, g = w % G;
      for (int j = 0; j < K; ++j)
        for (int x = 0; x < L; ++x) {
          const int z = g + j * G;
          const int p = j * L + x;
          const int i = x + L * (y + L * z);
          const int ixm = ((x + L - 1) % L) + L * (y + L * z);
          const int iym = x + L * (((y + L - 1) % L) + L * z);
          const int izm = x + L * (y + L * ((z + L - 1) % L));
          const int8_t jv[6] = {J[i], J[ixm], J[N + i], J[N + iym], J[2 * N + i], J[2 * N + izm]};
          for (int d = 0; d < 6; ++d)
            if (jv[d] < 0) m[d] |= 1u << p;
        }
    }
    for (int d = 0; d < 6; ++d) bonds[d * W + w] = m[d];
  }
}

// Coupling / presence masks of a chain from int8 J[N] (J[N-1] = wrap bond).
__global__ void k_setup_bonds1d(const int8_t* __restrict__ J, int N, int W,
                                uint32_t* __restrict__ bonds) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += gridDim.x * blockDim.x) {
    uint32_t jp = 0, jm = 0, pp = 0, pm = 0;
    for (int p = 0; p < 32; ++p) {
      const int i = 32 * w + p;
      if (i >= N) break;
      const int8_t a = J[i], b = J[(i + N - 1) % N];
      if (a < 0) jp |= 1u << p;
      if (b < 0) jm |= 1u << p;
      if (a != 0) pp |= 1u << p;
      if (b != 0) pm |= 1u << p;
    }
    bonds[0 * W + w] = jp;
    bonds[1 * W + w] = jm;
    bonds[2 * W + w] = pp;
    bonds[3 * W + w] = pm;
  }
}

// beta = 0 state before the init kernel fills the population (Sec. 2: ln Omega).
__global__ void k_init_state(RunDev* __restrict__ runs, const int32_t* __restrict__ ids, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  RunDev& R = runs[ids ? ids[t] : t];
  R.cur = 0;
  R.error = 0;
  R.skip = 0;
  R.step = 0;
  R.sweeps = 0;
  R.beta = 0.0;
  R.mbF = __dmul_rn((double)R.N, LN2_NEAREST);
  R.lnQ_last = 0.0;
  R.Qp_last = 0.0;
  R.sumE_next = 0ull;
  R.sumE2_next = 0ull;
  R.emin_next = 0x7FFFFFFFFFFFFFFFll;
  R.sumE2hi_next = 0ull;
  R.R_next = R.R;
}

__global__ void k_zero_hist(RunDev* __restrict__ runs, const int32_t* __restrict__ ids, int n, int which) {
  const int t = blockIdx.y;
  if (t >= n) return;
  RunDev& R = runs[ids ? ids[t] : t];
  uint32_t* h = R.hist[which];
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < R.nbins; b += gridDim.x * blockDim.x) h[b] = 0u;
}

// Energy sums of the measured population become the committed ones.  The
// Gaussian model's record keeps the bits of the physical sum of E^2 in the
// sumE2 slot (the integer sum does not fit 64 bits).
__device__ __forceinline__ void commit_energy_sums(RunDev& R) {
  R.sumE = (int64_t)R.sumE_next;
  R.sumE2 = (int64_t)R.sumE2_next;
  R.emin = R.emin_next;
  if (R.model == 1) {
    const double s = __dadd_rn(__dmul_rn((double)R.sumE2hi_next, 4294967296.0), (double)R.sumE2_next);
    R.sumE2d = __dmul_rn(s, 0x1.0p-30);
    R.sumE2 = __double_as_longlong(R.sumE2d);
  }
}

__global__ void k_init_finish(RunDev* __restrict__ runs, const int32_t* __restrict__ ids, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  RunDev& R = runs[ids ? ids[t] : t];
  commit_energy_sums(R);
  R.rec_beta[0] = 0.0;
  R.rec_lnQ[0] = 0.0;
  R.rec_mbF[0] = R.mbF;
  R.rec_R[0] = R.R;
  R.rec_sumE[0] = R.sumE;
  R.rec_sumE2[0] = R.sumE2;
}

// ---------------------------------------------------------------------------
// Step: Q, ln Q, -beta F~, Poisson tables, thresholds (one warp per run)
// ---------------------------------------------------------------------------
constexpr int PREP_THREADS = 256;
constexpr int PREP_WIN = 2048;  // bins of one shared-memory window of the Q' sum

// Every FP64 instruction holds an SM sub-partition for about 64 cycles on
// this GPU, so the kernel keeps the FP64 chains short and side by side: the
// per-bin work is spread over the block, the Q' tree reads its terms from
// shared memory and visits only the occupied range of bins, and ln Q and the
// thresholds are computed by threads without bins while the others build the
// Poisson tables.
__global__ void __launch_bounds__(PREP_THREADS) k_prepare(RunDev* __restrict__ runs,
                                                          const int32_t* __restrict__ ids, int use_override,
                                                          double beta_o, int theta_o, int64_t Rt_o) {
  __shared__ int s_ok, s_bmin, s_bmax, s_theta, s_nocc;
  __shared__ double s_bn, s_Qp;
  __shared__ long long s_Rt;
  __shared__ double s_term[PREP_WIN];
  RunDev& R = runs[ids ? ids[blockIdx.x] : blockIdx.x];
  const int tid = threadIdx.x;
  if (tid == 0) {
    int ok = 1;
    double bn = 0.0;
    int th = 0;
    int64_t Rt = 0;
    if (R.error) {
      ok = 0;
    } else if (use_override) {
      bn = beta_o < 0.0 ? R.beta : beta_o;
      th = theta_o;
      Rt = Rt_o < 0 ? R.R : Rt_o;
    } else if (R.step >= R.n_sched || R.step >= R.max_steps) {
      ok = 0;  // schedule exhausted: the run is finished, nothing to do
    } else {
      bn = R.sched_beta[R.step];
      th = R.sched_theta[R.step];
      Rt = R.sched_R[R.step];
    }
    if (ok && (!(bn >= R.beta) || th < 0 || Rt < 1)) {
      R.error = ERR_INVALID;
      ok = 0;
    }
    if (!ok) R.skip = 1;
    s_ok = ok;
    s_bn = bn;
    s_theta = th;
    s_Rt = Rt;
    s_bmin = 0x7FFFFFFF;
    s_bmax = -1;
    s_nocc = 0;
  }
  __syncthreads();
  if (!s_ok) return;
  const double bn = s_bn;
  const int64_t Rt = s_Rt;
  const double dbeta = __dsub_rn(bn, R.beta);
  const uint32_t* __restrict__ h = R.hist[R.cur];
  const int nbins = R.nbins;
  double* __restrict__ w = R.bin_w;

  // occupied bins, compacted so the FP64 work below spreads evenly over the
  // block; the first and last occupied bins
  int32_t* __restrict__ occ = R.occ;
  for (int b = tid; b < nbins; b += PREP_THREADS)
    if (h[b] != 0u) {
      atomicMin(&s_bmin, b);
      atomicMax(&s_bmax, b);
      occ[atomicAdd(&s_nocc, 1)] = b;
    }
  __syncthreads();
  const int bmin = s_bmin, bmax = s_bmax;
  const int nocc = s_nocc;
  // reweighting factors of the occupied bins, w_b = exp(-dbeta (E_b - E_min))
  for (int i = tid; i < nocc; i += PREP_THREADS) {
    const int b = occ[i];
    w[b] = dexp_np(-__dmul_rn(dbeta, (double)(2 * (b - bmin))));
  }
  __syncthreads();
  // Q' = sum_b n_b w_b over the fixed tree: lane l sums the terms of bins
  // l, l+32, ... in increasing order, then butterfly levels 16, 8, 4, 2, 1.
  // An empty bin adds +0.0, which leaves the sum unchanged, so the lanes may
  // run over whole windows of the occupied range [bmin, bmax].
  double acc = 0.0;
  for (int lo = bmin & ~31; lo <= bmax; lo += PREP_WIN) {
    const int span = min(PREP_WIN, bmax + 1 - lo);
    for (int t = tid; t < span; t += PREP_THREADS) s_term[t] = 0.0;
    __syncthreads();
    for (int i = tid; i < nocc; i += PREP_THREADS) {
      const int b = occ[i];
      if (b >= lo && b < lo + span) s_term[b - lo] = __dmul_rn((double)h[b], w[b]);
    }
    __syncthreads();
    if (tid < 32)
      for (int t = tid; t < span; t += 32) acc = __dadd_rn(acc, s_term[t]);
    __syncthreads();
  }
  if (tid < 32) {
#pragma unroll
    for (int sh = 16; sh >= 1; sh >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, sh));
    if (tid == 0) s_Qp = acc;
  }
  __syncthreads();
  const double Qp = s_Qp;
  // ln Q, the staged -beta F~ and the thresholds by the last threads, which
  // have no bin while nocc < PREP_THREADS - 8
  if (tid == PREP_THREADS - 1) {
    const int64_t Emin = 2 * (int64_t)bmin - R.Nb;
    const double lnQ = __dsub_rn(__dsub_rn(log(Qp), log((double)R.R)), __dmul_rn(dbeta, (double)Emin));
    R.lnQ_staged = lnQ;
    R.Qp_staged = Qp;
    R.mbF_staged = __dadd_rn(R.mbF, lnQ);
    R.beta_next = bn;
    R.theta_next = s_theta;
    R.Rt_next = Rt;
    R.bmin = bmin;
    R.sumE_next = 0ull;
    R.sumE2_next = 0ull;
    R.skip = 0;
  }
  if (tid >= PREP_THREADS - 9 && tid < PREP_THREADS - 1) {
    const int d = tid - (PREP_THREADS - 9);
    R.thr[d] = (d == 0 || d == 7) ? 0u : metropolis_threshold(bn, 2 * d);
  }
  // Poisson means a_b = R_target w_b / Q' = (R/R~) tau_j (Eq. (1)), split in
  // m = ceil(a/32) pieces when a > 32 (a / 32 and a / 1 are exact, so they
  // are taken as a product and as a itself).
  const double Rtd = (double)Rt;
  for (int i = tid; i < nocc; i += PREP_THREADS) {
    const int b = occ[i];
    const double a = __ddiv_rn(__dmul_rn(Rtd, w[b]), Qp);
    int64_t m = 1;
    double am = a;
    if (a > 32.0) {
      m = (int64_t)ceil(__dmul_rn(a, 0.03125));
      am = __ddiv_rn(a, (double)m);
    }
    const double p0 = dexp_np(-am);
    R.bin_am[b] = am;
    R.bin_p0[b] = p0;
    R.bin_m[b] = m;
    // the first POISSON_TAB partial sums C_k of the walk as 53-bit integer
    // thresholds (u >= C_k iff U >= ceil(C_k 2^53), u = U 2^-53), built with
    // the walk's own recurrence, and the state after the last of them
    uint64_t* tb = R.bin_thr + (size_t)b * POISSON_TAB;
    double P = p0, C = p0;
    tb[0] = cdf_threshold(C);
#pragma unroll 1
    for (int k = 1; k < POISSON_TAB; ++k) {
      P = div_small_rn(__dmul_rn(P, am), (uint32_t)k);
      C = __dadd_rn(C, P);
      tb[k] = cdf_threshold(C);
    }
    R.bin_end[2 * b] = P;
    R.bin_end[2 * b + 1] = C;
  }
  uint32_t* hn = R.hist[R.cur ^ 1];
  for (int b = tid; b < nbins; b += PREP_THREADS) hn[b] = 0u;
}

// ---------------------------------------------------------------------------
// Step: Poisson copy counts (Sec. 2: N[(R/R~) tau_j] copies of replica j)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t block_sum_i64(int64_t v, int64_t* s_warp) {
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, sh);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s_warp[wid] = v;
  __syncthreads();
  int64_t t = 0;
  if (threadIdx.x < 32) {
    t = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
#pragma unroll
    for (int sh = 16; sh >= 1; sh >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, sh);
  }
  return t;  // valid in thread 0
}

// Exclusive block scan (int64); returns the exclusive prefix, *total in all threads.
__device__ __forceinline__ int64_t block_exscan_i64(int64_t v, int64_t* s_warp, int64_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int sh = 1; sh < 32; sh <<= 1) {
    const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, sh);
    if (lane >= sh) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t s = (lane < nw) ? s_warp[lane] : 0;
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, s, sh);
      if (lane >= sh) s += y;
    }
    if (lane < nw) s_warp[lane] = s;  // inclusive warp totals
  }
  __syncthreads();
  const int64_t before = (wid > 0) ? s_warp[wid - 1] : 0;
  *total = s_warp[nw - 1];
  __syncthreads();
  return before + x - v;
}

// Inverse-CDF walk of one Poisson piece (mean am, P(0) = p0) for uniform u:
// P_k = (P_{k-1} am) / k, C_k = C_{k-1} + P_k, stop at the first k with
// u < C_k (or at POISSON_KMAX).  The division by k is the exact integer one
// of div_small_rn, the same double as a correctly rounded division.
__device__ __forceinline__ int poisson_piece(double u, double am, double p0) {
  int k = 0;
  double P = p0, C = p0;
  while (u >= C && k < POISSON_KMAX) {
    k = k + 1;
    P = div_small_rn(__dmul_rn(P, am), (uint32_t)k);
    C = __dadd_rn(C, P);
  }
  return k;
}

__device__ __forceinline__ int64_t pieces_sum(const RunDev& R, int64_t j, int64_t first, int64_t stride, int64_t m,
                                              double am, double p0) {
  const uint32_t stp = (uint32_t)R.step;
  int64_t c = 0;
  for (int64_t piece = first; piece < m; piece += stride) {
    const u32x4 r = philox_seeded(R.seed, (uint32_t)piece, (uint32_t)j, stp, TAG_RESAMPLE);
    c += poisson_piece(u53(r.a, r.b), am, p0);
  }
  return c;
}

// The same walk from a bin's table: with U the 53-bit integer of the
// uniform, the walk stops at the first k with U < thr[k]; the thresholds do
// not decrease, so that k is the number of thresholds U reaches.  Past the
// table the walk goes on from the stored state, step by step as above.
__device__ __forceinline__ int poisson_piece_tab(uint64_t U, const uint64_t* __restrict__ thr, double P, double C,
                                                 double am) {
  const ulonglong2* t2 = reinterpret_cast<const ulonglong2*>(thr);
  int k = 0;
#pragma unroll
  for (int q = 0; q < POISSON_TAB / 2; ++q) {
    const ulonglong2 v = t2[q];
    k += (U >= v.x) + (U >= v.y);
  }
  if (k < POISSON_TAB) return k;
  const double u = __dmul_rn((double)U, 0x1.0p-53);
  k = POISSON_TAB - 1;
  while (u >= C && k < POISSON_KMAX) {
    k = k + 1;
    P = div_small_rn(__dmul_rn(P, am), (uint32_t)k);
    C = __dadd_rn(C, P);
  }
  return k;
}

__device__ __forceinline__ int64_t pieces_sum_tab(const RunDev& R, int64_t j, int64_t first, int64_t stride,
                                                  int64_t m, int b) {
  const uint32_t stp = (uint32_t)R.step;
  const uint64_t* thr = R.bin_thr + (size_t)b * POISSON_TAB;
  int64_t c = 0;
  for (int64_t piece = first; piece < m; piece += stride) {
    const u32x4 r = philox_seeded(R.seed, (uint32_t)piece, (uint32_t)j, stp, TAG_RESAMPLE);
    const uint64_t U = ((((uint64_t)r.a) << 32) | (uint64_t)r.b) >> 11;
    c += poisson_piece_tab(U, thr, R.bin_end[2 * b], R.bin_end[2 * b + 1], R.bin_am[b]);
  }
  return c;
}

// Poisson pieces of replica j: from the per-bin tables (+-1 couplings) or
// from the replica's own weight (Gaussian couplings; same arithmetic as the
// per-bin tables of k_prepare).
__device__ __forceinline__ void replica_poisson(RunDev& R, int64_t j, int64_t* m, double* am, double* p0) {
  if (R.model == 0) {
    const int b = (R.E[R.cur][j] + R.Nb) >> 1;
    *m = R.bin_m[b];
    *am = R.bin_am[b];
    *p0 = R.bin_p0[b];
    return;
  }
  double a = __ddiv_rn(__dmul_rn((double)R.Rt_next, R.w_rep[j]), R.Qp_staged);
  // w_j <= Q' makes a <= R_target (up to rounding); anything else (a stale or
  // unset weight) draws nothing and flags the run instead of sampling an
  // unbounded mean
  if (!(a <= 2.0 * (double)R.Rt_next + 1.0)) {
    R.error = ERR_INVALID;
    a = 0.0;
  }
  int64_t mm = 1;
  double a1 = a;  // a / 1 and a / 32 are exact: taken as a itself and as a product
  if (a > 32.0) {
    mm = (int64_t)ceil(__dmul_rn(a, 0.03125));
    a1 = __ddiv_rn(a, (double)mm);
  }
  *m = mm;
  *am = a1;
  *p0 = dexp_np(-a1);
}

// Replicas whose mean needs more pieces than this are sampled by the whole
// block (pieces split over the threads, counts summed): after a large
// temperature step a few low-energy replicas carry most of the weight.
constexpr int64_t HEAVY_PIECES = 8;

__global__ void __launch_bounds__(CHUNK) k_copies(RunDev* __restrict__ runs, const Work* __restrict__ table) {
  __shared__ int64_t s_warp[CHUNK / 32];
  __shared__ int32_t s_heavy[CHUNK];
  __shared__ int s_nheavy;
  const Work wk = table[blockIdx.x];
  RunDev& R = runs[wk.run];
  if (R.skip) return;
  const int64_t j = (int64_t)wk.first + threadIdx.x;
  const int64_t Rold = R.R;
  if ((int64_t)wk.first >= Rold) {
    if (threadIdx.x == 0) R.chunk_sum[wk.first / CHUNK] = 0;
    return;
  }
  if (threadIdx.x == 0) s_nheavy = 0;
  __syncthreads();
  int64_t c = 0;
  if (j < Rold) {
    int64_t m;
    double am, p0;
    if (R.model == 0) {  // +-1 couplings: the bin's tables
      const int b = (R.E[R.cur][j] + R.Nb) >> 1;
      m = R.bin_m[b];
      if (m > HEAVY_PIECES) {
        s_heavy[atomicAdd(&s_nheavy, 1)] = (int32_t)(j - wk.first);
      } else {
        c = pieces_sum_tab(R, j, 0, 1, m, b);
        R.copies[j] = (int32_t)c;
      }
    } else {
      replica_poisson(R, j, &m, &am, &p0);
      if (m > HEAVY_PIECES) {
        s_heavy[atomicAdd(&s_nheavy, 1)] = (int32_t)(j - wk.first);
      } else {
        c = pieces_sum(R, j, 0, 1, m, am, p0);
        R.copies[j] = (int32_t)c;
      }
    }
  }
  __syncthreads();
  const int nh = s_nheavy;
  for (int h = 0; h < nh; ++h) {
    const int64_t jh = (int64_t)wk.first + s_heavy[h];
    int64_t mh;
    double amh, p0h;
    int64_t part;
    if (R.model == 0) {
      const int bh = (R.E[R.cur][jh] + R.Nb) >> 1;
      part = pieces_sum_tab(R, jh, threadIdx.x, CHUNK, R.bin_m[bh], bh);
    } else {
      replica_poisson(R, jh, &mh, &amh, &p0h);
      part = pieces_sum(R, jh, threadIdx.x, CHUNK, mh, amh, p0h);
    }
    const int64_t tot = block_sum_i64(part, s_warp);
    if (threadIdx.x == 0) {
      R.copies[jh] = (int32_t)(tot > 0x7FFFFFFF ? 0x7FFFFFFF : tot);
      c += tot;  // thread 0 carries the heavy totals into the chunk sum
    }
    __syncthreads();
  }
  const int64_t tot = block_sum_i64(c, s_warp);
  if (threadIdx.x == 0) R.chunk_sum[wk.first / CHUNK] = tot;
}

__global__ void __launch_bounds__(CHUNK) k_scan(RunDev* __restrict__ runs, const int32_t* __restrict__ ids) {
  __shared__ int64_t s_warp[CHUNK / 32];
  RunDev& R = runs[ids ? ids[blockIdx.x] : blockIdx.x];
  if (R.skip) return;
  const int nch = (int)((R.R + CHUNK - 1) / CHUNK);
  int64_t running = 0;
  for (int base = 0; base < nch; base += CHUNK) {
    const int i = base + threadIdx.x;
    const int64_t v = (i < nch) ? R.chunk_sum[i] : 0;
    int64_t tot;
    const int64_t ex = block_exscan_i64(v, s_warp, &tot);
    if (i < nch) R.chunk_off[i] = running + ex;
    running += tot;
  }
  if (threadIdx.x == 0) {
    R.R_next = running;
    if (running == 0) {
      R.error = ERR_EXTINCT;
      R.skip = 1;
    } else if (running > R.R_cap) {
      R.error = ERR_CAPACITY;
      R.skip = 1;
    }
  }
}

__global__ void __launch_bounds__(CHUNK) k_scatter(RunDev* __restrict__ runs, const Work* __restrict__ table) {
  __shared__ int64_t s_warp[CHUNK / 32];
  const Work wk = table[blockIdx.x];
  RunDev& R = runs[wk.run];
  if (R.skip) return;
  const int64_t Rold = R.R;
  if ((int64_t)wk.first >= Rold) return;
  const int64_t j = (int64_t)wk.first + threadIdx.x;
  const int64_t c = (j < Rold) ? R.copies[j] : 0;
  int64_t tot;
  const int64_t ex = block_exscan_i64(c, s_warp, &tot);
  const int64_t off = R.chunk_off[wk.first / CHUNK] + ex;
  for (int64_t q = 0; q < c; ++q) R.src[off + q] = (int32_t)j;
}

// Commit the step (or, after a device-detected error, leave the state as it was).
__global__ void k_commit(RunDev* __restrict__ runs, const int32_t* __restrict__ ids, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  RunDev& R = runs[ids ? ids[t] : t];
  if (R.skip || R.error) return;
  R.cur ^= 1;
  R.R = R.R_next;
  R.beta = R.beta_next;
  R.mbF = R.mbF_staged;
  R.lnQ_last = R.lnQ_staged;
  R.Qp_last = R.Qp_staged;
  R.step += 1;
  R.sweeps += R.theta_next;
  commit_energy_sums(R);
  const int64_t k = R.step;
  if (k <= R.max_steps) {
    R.rec_beta[k] = R.beta;
    R.rec_lnQ[k] = R.lnQ_last;
    R.rec_mbF[k] = R.mbF;
    R.rec_R[k] = R.R;
    R.rec_sumE[k] = R.sumE;
    R.rec_sumE2[k] = R.sumE2;
  }
}

// ---------------------------------------------------------------------------
// Read-out
// ---------------------------------------------------------------------------
__device__ __forceinline__ void site_word_bit(const RunDev& R, int64_t i, int* w, int* p) {
  if (R.dim == 1) {
    *w = (int)(i >> 5);
    *p = (int)(i & 31);
    return;
  }
  const int Lx = R.bx > 0 ? R.bx : R.L, Ly = R.bx > 0 ? R.by : R.L, Lz = R.bx > 0 ? R.bz : R.L;
  const int K = R.bx > 0 ? R.bk : lanes_for(R.L), G = Lz / K;
  const int x = (int)(i % Lx), y = (int)((i / Lx) % Ly), z = (int)(i / ((int64_t)Lx * Ly));
  *w = y * G + z % G;
  *p = (z / G) * Lx + x;
}

// Spins of slots [0, n) as int8 +-1 in natural site order.
__global__ void k_unpack(const RunDev* __restrict__ runs, int r, int64_t n, int8_t* __restrict__ out) {
  const RunDev& R = runs[r];
  const int64_t total = n * (int64_t)R.N;
  const uint32_t* sp = R.spins[R.cur];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / R.N, i = t % R.N;
    int w, p;
    site_word_bit(R, i, &w, &p);
    const uint32_t bit = (sp[s * R.W + w] >> p) & 1u;
    out[t] = bit ? (int8_t)-1 : (int8_t)1;
  }
}

// Sec. 4 overlap: replica k of run a against replica k of run b.
__global__ void k_overlap(const RunDev* __restrict__ pa_, const RunDev* __restrict__ pb_, double qcut,
                          unsigned long long* __restrict__ count, unsigned long long* __restrict__ hist) {
  const RunDev& A = *pa_;
  const RunDev& B = *pb_;
  const int64_t n = A.R < B.R ? A.R : B.R;
  const int W = A.W;
  const double lim = __dmul_rn(qcut, (double)A.N);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t* a = A.spins[A.cur] + k * W;
    const uint32_t* b = B.spins[B.cur] + k * W;
    int diff = 0;
    for (int w = 0; w < W; ++w) diff += __popc(a[w] ^ b[w]);
    const int dot = A.N - 2 * diff;
    if (fabs((double)dot) < lim) atomicAdd(count, 1ull);
    if (hist) atomicAdd(&hist[(dot + A.N) >> 1], 1ull);
  }
}

// Sec. 4 overlap for many pairs of runs of one batch at once: pair p counts
// the replicas k < min(R~_a, R~_b) with |q_k| < qcut, q_k the overlap of
// replica k of run ra[p] with replica k of run rb[p] (blockIdx.y = pair).
__global__ void k_overlap_pairs(const RunDev* __restrict__ runs, const int32_t* __restrict__ ra,
                                const int32_t* __restrict__ rb, int n_pairs, double qcut,
                                unsigned long long* __restrict__ count) {
  const int p = blockIdx.y;
  if (p >= n_pairs) return;
  const RunDev& A = runs[ra[p]];
  const RunDev& B = runs[rb[p]];
  const int64_t n = A.R < B.R ? A.R : B.R;
  const int W = A.W;
  const double lim = __dmul_rn(qcut, (double)A.N);
  unsigned long long local = 0ull;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t* a = A.spins[A.cur] + k * W;
    const uint32_t* b = B.spins[B.cur] + k * W;
    int diff = 0;
    for (int w = 0; w < W; ++w) diff += __popc(a[w] ^ b[w]);
    const int dot = A.N - 2 * diff;
    if (fabs((double)dot) < lim) ++local;
  }
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) local += __shfl_xor_sync(0xFFFFFFFFu, local, sh);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(&count[p], local);
}

// Histogram of the overlap for each pair of runs (Sec. 4, P(q)): bin
// (N q + N) / 2 = N - (sites that differ) of replica k of run ra[p] against
// replica k of run rb[p], k < min(R~_a, R~_b), counted in shared memory
// (N + 1 bins) and added to hist[p][.].
__global__ void k_overlap_hist(const RunDev* __restrict__ runs, const int32_t* __restrict__ ra,
                               const int32_t* __restrict__ rb, int n_pairs, int nbins,
                               unsigned long long* __restrict__ hist) {
  extern __shared__ uint32_t s_bins[];
  const int p = blockIdx.y;
  if (p >= n_pairs) return;
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) s_bins[i] = 0u;
  __syncthreads();
  const RunDev& A = runs[ra[p]];
  const RunDev& B = runs[rb[p]];
  const int64_t n = A.R < B.R ? A.R : B.R;
  const int W = A.W, N = A.N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t* a = A.spins[A.cur] + k * W;
    const uint32_t* b = B.spins[B.cur] + k * W;
    int diff = 0;
    for (int w = 0; w < W; ++w) diff += __popc(a[w] ^ b[w]);
    const int bin = N - diff;  // unused bits of the words are zero, so 0 <= bin <= N
    if (bin >= 0) atomicAdd(&s_bins[bin], 1u);
  }
  __syncthreads();
  unsigned long long* hp = hist + (size_t)p * nbins;
  for (int i = threadIdx.x; i < nbins; i += blockDim.x)
    if (s_bins[i]) atomicAdd(&hp[i], (unsigned long long)s_bins[i]);
}

cudaError_t launch_overlap_hist(const RunDev* runs, const int32_t* ra, const int32_t* rb, int n_pairs, int nbins,
                                unsigned long long* hist, cudaStream_t st) {
  if (n_pairs <= 0) return cudaSuccess;
  dim3 grid(16, n_pairs);
  k_overlap_hist<<<grid, 256, sizeof(uint32_t) * (size_t)nbins, st>>>(runs, ra, rb, n_pairs, nbins, hist);
  return cudaGetLastError();
}

cudaError_t launch_overlap_pairs(const RunDev* runs, const int32_t* ra, const int32_t* rb, int n_pairs, double qcut,
                                 unsigned long long* count, cudaStream_t st) {
  if (n_pairs <= 0) return cudaSuccess;
  dim3 grid(16, n_pairs);
  k_overlap_pairs<<<grid, 256, 0, st>>>(runs, ra, rb, n_pairs, qcut, count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sec. 3 weighted averages: one warp per group of M runs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, sh));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xFFFFFFFFu, v, sh));
  return v;
}

// PAIRS: Sec. 4, Eq. (11) -- an observable of two independent runs
// (the overlap) is averaged over M pairs with weights e^{-beta (F~1 + F~2)}
// (R1 R2 e^{...} with the population factors of Eq. (6)), and fbar is
// ln[(1/M) sum_r e^{x1_r + x2_r}].  Otherwise x2 and Rw2 are unused.
template <bool PAIRS>
__global__ void __launch_bounds__(32) k_weighted(int M, const double* __restrict__ x, const double* __restrict__ x2,
                                                 const double* __restrict__ A, const double* __restrict__ Rw,
                                                 const double* __restrict__ Rw2, double* __restrict__ mean,
                                                 double* __restrict__ fbar) {
  const int g = blockIdx.x, lane = threadIdx.x;
  const double* xg = x + (int64_t)g * M;
  const double* x2g = PAIRS ? x2 + (int64_t)g * M : nullptr;
  const double* Ag = A ? A + (int64_t)g * M : nullptr;
  const double* Rg = Rw ? Rw + (int64_t)g * M : nullptr;
  const double* R2g = (PAIRS && Rw2) ? Rw2 + (int64_t)g * M : nullptr;
  auto xr = [&](int r) { return PAIRS ? xg[r] + x2g[r] : xg[r]; };
  auto yr = [&](int r) {
    double y = xr(r);
    if (Rg) y = y + log(Rg[r]);
    if (PAIRS && R2g) y = y + log(R2g[r]);
    return y;
  };
  double mu = -INFINITY, mux = -INFINITY;
  for (int r = lane; r < M; r += 32) {
    mu = fmax(mu, yr(r));
    mux = fmax(mux, xr(r));
  }
  mu = warp_max(mu);
  mux = warp_max(mux);
  double S = 0.0, SA = 0.0, Sx = 0.0;
  for (int r = lane; r < M; r += 32) {
    const double e = exp(yr(r) - mu);
    S += e;
    if (Ag) SA += e * Ag[r];
    Sx += exp(xr(r) - mux);
  }
  S = warp_sum(S);
  SA = warp_sum(SA);
  Sx = warp_sum(Sx);
  if (lane == 0) {
    mean[g] = Ag ? SA / S : 0.0;
    fbar[g] = mux + log(Sx) - log((double)M);
  }
}

// Sec. 3 bootstrap: resample b draws index floor(word0 * M / 2^32) of
// Philox(ctr = (b, i, 0, TAG_BOOT)); one thread per resample.  GK groups of M
// values each (x, A, Rw laid out [GK][M]) are resampled with the same draws;
// the results are laid out [GK][B].
__global__ void k_bootstrap(int M, const double* __restrict__ x, const double* __restrict__ A,
                            const double* __restrict__ Rw, int B, uint64_t seed, int GK,
                            double* __restrict__ bmean, double* __restrict__ bfbar) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  for (int gk = blockIdx.y; gk < GK; gk += gridDim.y) {
    const double* xg = x + (int64_t)gk * M;
    const double* Ag = A ? A + (int64_t)gk * M : nullptr;
    const double* Rg = Rw ? Rw + (int64_t)gk * M : nullptr;
    double mu = -INFINITY, mux = -INFINITY;
    for (int i = 0; i < M; ++i) {
      const u32x4 r = philox_seeded(seed, (uint32_t)b, (uint32_t)i, 0u, TAG_BOOT);
      const int k = (int)(((uint64_t)r.a * (uint64_t)M) >> 32);
      const double y = Rg ? xg[k] + log(Rg[k]) : xg[k];
      mu = fmax(mu, y);
      mux = fmax(mux, xg[k]);
    }
    double S = 0.0, SA = 0.0, Sx = 0.0;
    for (int i = 0; i < M; ++i) {
      const u32x4 r = philox_seeded(seed, (uint32_t)b, (uint32_t)i, 0u, TAG_BOOT);
      const int k = (int)(((uint64_t)r.a * (uint64_t)M) >> 32);
      const double y = Rg ? xg[k] + log(Rg[k]) : xg[k];
      const double e = exp(y - mu);
      S += e;
      if (Ag) SA += e * Ag[k];
      Sx += exp(xg[k] - mux);
    }
    bmean[(int64_t)gk * B + b] = Ag ? SA / S : 0.0;
    bfbar[(int64_t)gk * B + b] = mux + log(Sx) - log((double)M);
  }
}

// Self-check of div_small_rn: n pairs (x, k) with x from 63 random bits
// (every exponent, zero, subnormals, infinities and NaNs) and k uniform in
// 1..POISSON_KMAX, each compared bit for bit with the division instruction;
// the number of differing pairs is added to *mismatches.
__global__ void k_check_division(int64_t n, uint64_t seed, unsigned long long* __restrict__ mismatches) {
  unsigned long long bad = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const u32x4 r = philox_seeded(seed, (uint32_t)i, (uint32_t)(i >> 32), 0u, 0x44495643u);
    const uint64_t bits = ((((uint64_t)r.a) << 32) | r.b) & 0x7FFFFFFFFFFFFFFFull;
    // half of the draws keep the exponent within 2^-60..2^6, where the walk's
    // terms P_k am live
    const uint64_t xb = (r.d & 1u) ? bits : ((bits & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(963 + r.d % 67u) << 52));
    const double x = __longlong_as_double((long long)xb);
    const uint32_t k = 1u + r.c % (uint32_t)POISSON_KMAX;
    const double q = div_small_rn(x, k), qd = __ddiv_rn(x, (double)k);
    if (__double_as_longlong(q) != __double_as_longlong(qd)) bad += 1ull;
  }
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) bad += __shfl_xor_sync(0xFFFFFFFFu, bad, sh);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(mismatches, bad);
}

// Self-check of the deterministic exponentials against CUDA's exp and expf:
// n seeded points, x uniform in [-745, 0] for dexp_np and in [-103, 0] for
// fexp_np; the largest distance in units in the last place of the CUDA value
// (both are finite and positive there; zero results count as 0 ulp apart
// only if both are zero).  out[0] = max ulp of dexp_np, out[1] = of fexp_np.
__device__ __forceinline__ unsigned long long ulp_distance_d(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return (unsigned long long)(ia > ib ? ia - ib : ib - ia);  // same sign, finite
}

__global__ void k_check_exp(int64_t n, uint64_t seed, unsigned long long* __restrict__ out) {
  unsigned long long md = 0ull, mf = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const u32x4 r = philox_seeded(seed, (uint32_t)i, (uint32_t)(i >> 32), 0u, 0x45585043u);
    const double xd = -745.0 * u53(r.a, r.b);
    const float xf = -103.0f * ((float)(r.c >> 8) * 0x1.0p-24f);
    md = max(md, ulp_distance_d(dexp_np(xd), exp(xd)));
    const int fa = __float_as_int(fexp_np(xf)), fb = __float_as_int(expf(xf));
    mf = max(mf, (unsigned long long)(fa > fb ? fa - fb : fb - fa));
  }
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) {
    md = max(md, __shfl_xor_sync(0xFFFFFFFFu, md, sh));
    mf = max(mf, __shfl_xor_sync(0xFFFFFFFFu, mf, sh));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], md);
    atomicMax(&out[1], mf);
  }
}

cudaError_t launch_check_exp(int64_t n, uint64_t seed, unsigned long long* out, cudaStream_t st) {
  k_check_exp<<<152 * 4, 256, 0, st>>>(n, seed, out);
  return cudaGetLastError();
}

cudaError_t launch_check_division(int64_t n, uint64_t seed, unsigned long long* mismatches, cudaStream_t st) {
  k_check_division<<<152 * 8, 256, 0, st>>>(n, seed, mismatches);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
cudaError_t set_exp_coefficients() {
  double c[DEXP_DEGREE + 1];
  c[0] = 1.0;
  for (int j = 1; j <= DEXP_DEGREE; ++j) c[j] = c[j - 1] / (double)j;
  cudaError_t e = cudaMemcpyToSymbol(c_dexp_coef, c, sizeof c);
  if (e != cudaSuccess) return e;
  // reciprocals floor(2^64 / k) of div_small_rn: (2^64 - 1) div k, plus one
  // where k divides 2^64
  uint64_t r[POISSON_KMAX + 1] = {0u, 0u};
  for (uint64_t k = 2; k <= (uint64_t)POISSON_KMAX; ++k) r[k] = ~0ull / k + ((~0ull % k) == k - 1u ? 1u : 0u);
  return cudaMemcpyToSymbol(c_recip_k, r, sizeof r);
}

cudaError_t launch_setup_bonds3d(const int8_t* J, int L, uint32_t* bonds, int W, cudaStream_t st) {
  const int K = lanes_for(L), G = L / K;
  k_setup_bonds3d<<<(W + 127) / 128, 128, 0, st>>>(J, L, K, G, W, bonds);
  return cudaGetLastError();
}
cudaError_t launch_setup_bonds1d(const int8_t* J, int N, uint32_t* bonds, int W, cudaStream_t st) {
  k_setup_bonds1d<<<(W + 127) / 128, 128, 0, st>>>(J, N, W, bonds);
  return cudaGetLastError();
}
cudaError_t launch_init_state(RunDev* runs, const int32_t* ids, int n, int max_bins, cudaStream_t st) {
  k_init_state<<<(n + 127) / 128, 128, 0, st>>>(runs, ids, n);
  dim3 g((max_bins + 255) / 256, n);
  k_zero_hist<<<g, 256, 0, st>>>(runs, ids, n, 0);
  return cudaGetLastError();
}
cudaError_t launch_init_finish(RunDev* runs, const int32_t* ids, int n, cudaStream_t st) {
  k_init_finish<<<(n + 127) / 128, 128, 0, st>>>(runs, ids, n);
  return cudaGetLastError();
}
cudaError_t launch_prepare(RunDev* runs, const int32_t* ids, int n, bool ovr, double beta, int theta,
                           int64_t Rt, cudaStream_t st) {
  k_prepare<<<n, PREP_THREADS, 0, st>>>(runs, ids, ovr ? 1 : 0, beta, theta, Rt);
  return cudaGetLastError();
}
cudaError_t launch_copies(RunDev* runs, const Work* table, int nwork, cudaStream_t st) {
  k_copies<<<nwork, CHUNK, 0, st>>>(runs, table);
  return cudaGetLastError();
}
cudaError_t launch_scan(RunDev* runs, const int32_t* ids, int n, cudaStream_t st) {
  k_scan<<<n, CHUNK, 0, st>>>(runs, ids);
  return cudaGetLastError();
}
cudaError_t launch_scatter(RunDev* runs, const Work* table, int nwork, cudaStream_t st) {
  k_scatter<<<nwork, CHUNK, 0, st>>>(runs, table);
  return cudaGetLastError();
}
cudaError_t launch_commit(RunDev* runs, const int32_t* ids, int n, cudaStream_t st) {
  k_commit<<<(n + 127) / 128, 128, 0, st>>>(runs, ids, n);
  return cudaGetLastError();
}
cudaError_t launch_unpack(const RunDev* runs, int r, int64_t n, int8_t* out, cudaStream_t st) {
  k_unpack<<<1216, 256, 0, st>>>(runs, r, n, out);
  return cudaGetLastError();
}
cudaError_t launch_overlap(const RunDev* a, const RunDev* b, double qcut, unsigned long long* count,
                           unsigned long long* hist, cudaStream_t st) {
  k_overlap<<<608, 256, 0, st>>>(a, b, qcut, count, hist);
  return cudaGetLastError();
}
// Per-step records of groups of M consecutive runs as [G][count][M] arrays:
// x = -beta F~, A = E_mean (physical units), Rw = the target population of
// the step that produced the record (R0 for the initial state).
__global__ void k_gather_records(const RunDev* __restrict__ runs, int M, int count, int G, double* __restrict__ x,
                                 double* __restrict__ A, double* __restrict__ Rw) {
  const int64_t total = (int64_t)G * count * M;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % M), k = (int)((t / M) % count), g = (int)(t / ((int64_t)M * count));
    const RunDev& R = runs[g * M + i];
    const double unit = R.model == 1 ? 0x1.0p-15 : 1.0;
    x[t] = R.rec_mbF[k];
    A[t] = __ddiv_rn(__dmul_rn((double)R.rec_sumE[k], unit), (double)R.rec_R[k]);
    Rw[t] = k == 0 ? (double)R.rec_R[0] : (double)R.sched_R[k - 1];
  }
}

// Var(x) over each group of M values (ddof 1), two passes (mean, then squared
// deviations), each summed lane-strided and by the butterfly; root = 1 gives
// the standard deviation instead.
__global__ void __launch_bounds__(32) k_variance(int M, const double* __restrict__ x, double* __restrict__ var,
                                                 int root) {
  const int g = blockIdx.x, lane = threadIdx.x;
  const double* xg = x + (int64_t)g * M;
  double s = 0.0;
  for (int r = lane; r < M; r += 32) s += xg[r];
  const double m = warp_sum(s) / (double)M;
  double v = 0.0;
  for (int r = lane; r < M; r += 32) v += (xg[r] - m) * (xg[r] - m);
  v = warp_sum(v);
  if (lane == 0) {
    const double w = M > 1 ? v / (double)(M - 1) : 0.0;
    var[g] = root ? sqrt(w) : w;
  }
}

cudaError_t launch_gather_records(const RunDev* runs, int M, int count, int G, double* x, double* A, double* Rw,
                                  cudaStream_t st) {
  const int64_t total = (int64_t)G * count * M;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  k_gather_records<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(runs, M, count, G, x, A, Rw);
  return cudaGetLastError();
}
cudaError_t launch_variance(int G, int M, const double* x, double* var, cudaStream_t st, bool root) {
  k_variance<<<G, 32, 0, st>>>(M, x, var, root ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_weighted(int G, int M, const double* x, const double* A, const double* Rw, double* mean,
                            double* fbar, cudaStream_t st) {
  k_weighted<false><<<G, 32, 0, st>>>(M, x, nullptr, A, Rw, nullptr, mean, fbar);
  return cudaGetLastError();
}
cudaError_t launch_weighted_pairs(int G, int M, const double* x1, const double* x2, const double* A,
                                  const double* R1, const double* R2, double* mean, double* fbar, cudaStream_t st) {
  k_weighted<true><<<G, 32, 0, st>>>(M, x1, x2, A, R1, R2, mean, fbar);
  return cudaGetLastError();
}
cudaError_t launch_bootstrap(int M, const double* x, const double* A, const double* Rw, int B, uint64_t seed,
                             double* bmean, double* bfbar, cudaStream_t st, int GK) {
  const dim3 grid((B + 127) / 128, (unsigned)std::min(GK, 65535));
  k_bootstrap<<<grid, 128, 0, st>>>(M, x, A, Rw, B, seed, GK, bmean, bfbar);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Gaussian couplings: Q' over replicas (fixed two-level tree)
//   level 1: chunk c of 256 slots: lane l sums w_j, j = 256c + l + 32i,
//            i = 0..7 (j < R~), in increasing i; butterfly 16, 8, 4, 2, 1;
//   level 2: lane l sums the chunk sums c = l, l+32, ... in increasing c;
//            butterfly 16, 8, 4, 2, 1.
// w_j = exp(-dbeta * (E_j - E_min) * 2^-15) with the deterministic exp.
// ---------------------------------------------------------------------------
__global__ void k_gprep_head(RunDev* __restrict__ runs, const int32_t* __restrict__ ids, int n, int use_override,
                             double beta_o, int theta_o, int64_t Rt_o) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  RunDev& R = runs[ids ? ids[t] : t];
  int ok = 1;
  double bn = 0.0;
  int th = 0;
  int64_t Rt = 0;
  if (R.error) {
    ok = 0;
  } else if (use_override) {
    bn = beta_o < 0.0 ? R.beta : beta_o;
    th = theta_o;
    Rt = Rt_o < 0 ? R.R : Rt_o;
  } else if (R.step >= R.n_sched || R.step >= R.max_steps) {
    ok = 0;
  } else {
    bn = R.sched_beta[R.step];
    th = R.sched_theta[R.step];
    Rt = R.sched_R[R.step];
  }
  if (ok && (!(bn >= R.beta) || th < 0 || Rt < 1)) {
    R.error = ERR_INVALID;
    ok = 0;
  }
  R.skip = ok ? 0 : 1;
  if (!ok) return;
  R.beta_next = bn;
  R.theta_next = th;
  R.Rt_next = Rt;
  R.sumE_next = 0ull;
  R.sumE2_next = 0ull;
  R.sumE2hi_next = 0ull;
  R.emin_next = 0x7FFFFFFFFFFFFFFFll;
}

__global__ void __launch_bounds__(CHUNK) k_gweights(RunDev* __restrict__ runs, const Work* __restrict__ table) {
  __shared__ double s_w[CHUNK];
  const Work wk = table[blockIdx.x];
  RunDev& R = runs[wk.run];
  if (R.skip) return;
  const int64_t Rold = R.R;
  if ((int64_t)wk.first >= Rold) return;
  const int64_t j = (int64_t)wk.first + threadIdx.x;
  const double dbeta = __dsub_rn(R.beta_next, R.beta);
  double w = 0.0;
  if (j < Rold) {
    const double de = __dmul_rn((double)((long long)R.E[R.cur][j] - R.emin), GAUSS_INV_SCALE_D);
    w = dexp_np(-__dmul_rn(dbeta, de));
    R.w_rep[j] = w;
  }
  s_w[threadIdx.x] = w;
  __syncthreads();
  if (threadIdx.x < 32) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < CHUNK / 32; ++i)
      if (wk.first + threadIdx.x + 32 * i < Rold) acc = __dadd_rn(acc, s_w[threadIdx.x + 32 * i]);
#pragma unroll
    for (int sh = 16; sh >= 1; sh >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, sh));
    if (threadIdx.x == 0) R.chunk_q[wk.first / CHUNK] = acc;
  }
}

__global__ void __launch_bounds__(32) k_gprep_tail(RunDev* __restrict__ runs, const int32_t* __restrict__ ids) {
  RunDev& R = runs[ids ? ids[blockIdx.x] : blockIdx.x];
  if (R.skip) return;
  const int lane = threadIdx.x;
  const int nch = (int)((R.R + CHUNK - 1) / CHUNK);
  double acc = 0.0;
  for (int c = lane; c < nch; c += 32) acc = __dadd_rn(acc, R.chunk_q[c]);
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, sh));
  if (lane == 0) {
    const double Qp = acc;
    const double dbeta = __dsub_rn(R.beta_next, R.beta);
    const double emin = __dmul_rn((double)R.emin, GAUSS_INV_SCALE_D);
    const double lnQ = __dsub_rn(__dsub_rn(log(Qp), log((double)R.R)), __dmul_rn(dbeta, emin));
    R.lnQ_staged = lnQ;
    R.Qp_staged = Qp;
    R.mbF_staged = __dadd_rn(R.mbF, lnQ);
  }
}

// Gaussian coupling tables of a 3D cubic lattice from int32 J[3][N]: for
// colour c, word w and rank m of the colour-c site in the word, the couplings
// of its six bonds (x+, x-, y+, y-, z+, z-) and their sum; ranks padded with
// zeros to SP, a multiple of 4.
__global__ void k_setup_gauss3d(const int32_t* __restrict__ J, int L, int K, int G, int32_t* __restrict__ gJ,
                                int32_t* __restrict__ gS) {
  const int WR = L * G, SITES = K * L / 2, SP = (SITES + 3) & ~3, N = L * L * L;
  const int total = 2 * WR * SP;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int m = t % SP, w = (t / SP) % WR, c = t / (SP * WR);
    int32_t v[6] = {0, 0, 0, 0, 0, 0};
    if (m < SITES) {
      const int j = m / (L / 2), xh = m % (L / 2);
      const int y = w / G, g = w % G, z = g + j * G;
      const int x = 2 * xh + ((c + y + z) & 1);
      const int i = x + L * (y + L * z);
      v[0] = J[i];
      v[1] = J[((x + L - 1) % L) + L * (y + L * z)];
      v[2] = J[N + i];
      v[3] = J[N + x + L * (((y + L - 1) % L) + L * z)];
      v[4] = J[2 * N + i];
      v[5] = J[2 * N + x + L * (y + L * ((z + L - 1) % L))];
    }
    int32_t sum = 0;
    for (int d = 0; d < 6; ++d) {
      gJ[((c * 6 + d) * WR + w) * SP + m] = v[d];
      sum += v[d];
    }
    gS[(c * WR + w) * SP + m] = sum;
  }
}

cudaError_t launch_setup_gauss3d(const int32_t* J, int L, int32_t* gJ, int32_t* gS, cudaStream_t st) {
  const int K = lanes_for(L), G = L / K;
  const int total = 2 * L * G * (((K * L / 2) + 3) & ~3);
  k_setup_gauss3d<<<(total + 255) / 256, 256, 0, st>>>(J, L, K, G, gJ, gS);
  return cudaGetLastError();
}
cudaError_t launch_gprep_head(RunDev* runs, const int32_t* ids, int n, bool ovr, double beta, int theta, int64_t Rt,
                              cudaStream_t st) {
  k_gprep_head<<<(n + 127) / 128, 128, 0, st>>>(runs, ids, n, ovr ? 1 : 0, beta, theta, Rt);
  return cudaGetLastError();
}
cudaError_t launch_gweights(RunDev* runs, const Work* table, int nwork, cudaStream_t st) {
  k_gweights<<<nwork, CHUNK, 0, st>>>(runs, table);
  return cudaGetLastError();
}
cudaError_t launch_gprep_tail(RunDev* runs, const int32_t* ids, int n, cudaStream_t st) {
  k_gprep_tail<<<n, 32, 0, st>>>(runs, ids);
  return cudaGetLastError();
}

}  // namespace pa
