// pa_gauss1d.cu -- fused replica copy + checkerboard Metropolis sweeps +
// energy measurement for chains with Gaussian couplings (Sec. 4: the periodic
// 1D spin glass the paper compares with exact transfer matrices).
//
// Bit p of word w of a replica is site 32 w + p; colour = site parity.  The
// couplings J_q[i] (bond i -> i+1, J_q[N-1] the wrap bond, 0 = absent) sit in
// shared memory as int32 and are read by every thread of the block at the
// same address (broadcast).  For site i with a+ = 1 where s_{i+1} != s_i and
// a- = 1 where s_{i-1} != s_i:
//   dE_i = 4 (a+ J[i] + a- J[i-1]) - 2 (J[i] + J[i-1]).
#include "pa_gauss.cuh"

namespace pa {

__device__ __forceinline__ uint32_t gchain_valid(int w, int WR, int nl) {
  return (w + 1 < WR || nl == 32) ? 0xFFFFFFFFu : ((1u << nl) - 1u);
}

// E_q = C0 - 2 sum over anti-aligned bonds (i, i+1) of J[i], C0 = sum J.
template <int TPB>
__device__ __forceinline__ int energy_gauss1d(const uint32_t* __restrict__ col, const int32_t* __restrict__ s_J,
                                              int WR, int nl, int32_t C0) {
  const uint32_t first = col[0];
  int32_t anti = 0;
  for (int w = 0; w < WR; ++w) {
    const uint32_t curw = col[w * TPB];
    const uint32_t nbp = (w + 1 < WR) ? __funnelshift_r(curw, col[(w + 1) * TPB], 1)
                                      : ((curw >> 1) | ((first & 1u) << (nl - 1)));
    uint32_t a = (curw ^ nbp) & gchain_valid(w, WR, nl);
    while (a) {
      anti += s_J[32 * w + __ffs(a) - 1];
      a &= a - 1u;
    }
  }
  return C0 - 2 * anti;
}

template <int TPB, int C>
__device__ __forceinline__ void half_sweep_gauss1d(uint32_t* __restrict__ col, const int32_t* __restrict__ s_J,
                                                   int N, int WR, int nl, uint32_t slot, uint32_t T,
                                                   const RoundKeys& rk, float beta_f, float bc, unsigned lanes,
                                                   uint32_t one) {
  constexpr uint32_t c = C;
  const uint32_t first = col[0];
  const uint32_t last = col[(WR - 1) * TPB];
  uint32_t prev = last, curw = first;
  const uint32_t tag = TAG_SWEEP + c;
#pragma unroll 1
  for (int w = 0; w < WR; ++w) {
    const uint32_t nextw = (w + 1 < WR) ? col[(w + 1) * TPB] : first;
    const uint32_t nbp = (w + 1 < WR) ? __funnelshift_r(curw, nextw, 1)
                                      : ((curw >> 1) | ((first & 1u) << (nl - 1)));
    const uint32_t nbm = (w > 0) ? __funnelshift_l(prev, curw, 1)
                                 : ((curw << 1) | ((last >> (nl - 1)) & 1u));
    const uint32_t ap = (curw ^ nbp) >> c, am = (curw ^ nbm) >> c;
    uint32_t u[16];
    const uint32_t ctr0 = (uint32_t)(w * 4);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const u32x4 v = philox10_rk(ctr0 + q, slot, T, tag, rk);
      u[4 * q + 0] = v.a;
      u[4 * q + 1] = v.b;
      u[4 * q + 2] = v.c;
      u[4 * q + 3] = v.d;
    }
    const int base = 32 * w + (int)c;
    // the word's 32 couplings (bond i -> i+1) in registers, four per 128-bit
    // load, and the one before them (the wrap bond J[N-1] for the first word);
    // past the chain's end they are the zero padding
    int32_t jv[33];
    jv[0] = (w > 0) ? s_J[32 * w - 1] : s_J[N - 1];
    const int4* J4 = reinterpret_cast<const int4*>(s_J + 32 * w);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int4 v = J4[q];
      jv[1 + 4 * q] = v.x;
      jv[2 + 4 * q] = v.y;
      jv[3 + 4 * q] = v.z;
      jv[4 + 4 * q] = v.w;
    }
    uint32_t flip = 0u, amb = 0u;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int32_t jp = jv[1 + C + 2 * m], jm = jv[C + 2 * m];
      int32_t acc = 0;
      add_if_set(acc, ap, 1u << (2 * m), jp, one);
      add_if_set(acc, am, 1u << (2 * m), jm, one);
      gauss_site(4 * acc - 2 * (jp + jm), bc, u[m], 1u << (2 * m), one, &flip, &amb);
    }
    amb &= (gchain_valid(w, WR, nl) >> C) & 0x55555555u;  // sites past the chain's end flip nothing
    if (__any_sync(lanes, amb != 0u)) {
      // sites inside the estimate's window: the exact decision, out of the
      // common path
      uint32_t a = amb;
      while (a) {
        const int bit = __ffs(a) - 1, m = bit >> 1;
        const int i = base + 2 * m;
        const int im = (i == 0) ? N - 1 : i - 1;
        const int32_t jp = s_J[i], jm = s_J[im];
        const int32_t acc = (((ap >> bit) & 1u) ? jp : 0) + (((am >> bit) & 1u) ? jm : 0);
        const u32x4 v = philox10_rk(ctr0 + (uint32_t)(m >> 2), slot, T, tag, rk);
        if (gauss_accept(4 * acc - 2 * (jp + jm), beta_f, pick(v, m & 3))) flip |= 1u << bit;
        a &= a - 1u;
      }
    }
    const uint32_t acc_mask = (flip << c) & gchain_valid(w, WR, nl);
    const uint32_t nw = curw ^ acc_mask;
    col[w * TPB] = nw;
    prev = nw;
    curw = nextw;
  }
}

__device__ __forceinline__ void measure_store_gauss1d(RunDev& R, int nxt, int64_t slot, bool live, int E) {
  long long e = 0ll;
  unsigned long long lo = 0ull, hi = 0ull;
  if (live) {
    R.E[nxt][slot] = E;
    atomicMin(&R.emin_next, (long long)E);
    e = E;
    const unsigned long long q = (unsigned long long)((long long)E * (long long)E);
    lo = q & 0xFFFFFFFFull;
    hi = q >> 32;
  }
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) {
    e += __shfl_xor_sync(0xFFFFFFFFu, e, sh);
    lo += __shfl_xor_sync(0xFFFFFFFFu, lo, sh);
    hi += __shfl_xor_sync(0xFFFFFFFFu, hi, sh);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&R.sumE_next, (unsigned long long)e);
    atomicAdd(&R.sumE2_next, lo);
    atomicAdd(&R.sumE2hi_next, hi);
  }
}

template <int TPB>
__global__ void __launch_bounds__(TPB) k_sweep_gauss1d(RunDev* __restrict__ runs, const Work* __restrict__ table,
                                                       int init) {
  extern __shared__ uint32_t smem[];
  const Work wk = table[blockIdx.x];
  RunDev& R = runs[wk.run];
  if (!init && R.skip) return;
  const int64_t Rn = init ? R.R : R.R_next;
  if ((int64_t)wk.first >= Rn) return;
  const int N = R.N, W = R.W, WR = R.Wr, nl = N - 32 * (WR - 1);
  int32_t* s_J = reinterpret_cast<int32_t*>(smem);
  uint32_t* s_spin = smem + 32 * WR;  // couplings padded to whole words
  const int tid = threadIdx.x;
  for (int i = tid; i < 32 * WR; i += TPB) s_J[i] = (i < N) ? R.gJ[i] : 0;
  const int64_t slot = (int64_t)wk.first + tid;
  const bool live = slot < Rn;
  const int cur = R.cur, nxt = init ? 0 : cur ^ 1;
  uint32_t* col = s_spin + tid;
  if (live) {
    if (init) {
      for (int w4 = 0; w4 < W / 4; ++w4) {
        const u32x4 u = philox_seeded(R.seed, (uint32_t)w4, (uint32_t)slot, 0u, TAG_INIT);
        const uint32_t v[4] = {u.a, u.b, u.c, u.d};
        for (int i = 0; i < 4; ++i) {
          const int w = 4 * w4 + i;
          if (w < WR) col[w * TPB] = v[i] & gchain_valid(w, WR, nl);
        }
      }
    } else {
      const int32_t src = R.src[slot];
      const uint4* p4 = reinterpret_cast<const uint4*>(R.spins[cur] + (size_t)src * W);
      for (int q = 0; q < W / 4; ++q) {
        const uint4 v = p4[q];
        if (4 * q + 0 < WR) col[(4 * q + 0) * TPB] = v.x;
        if (4 * q + 1 < WR) col[(4 * q + 1) * TPB] = v.y;
        if (4 * q + 2 < WR) col[(4 * q + 2) * TPB] = v.z;
        if (4 * q + 3 < WR) col[(4 * q + 3) * TPB] = v.w;
      }
    }
  }
  __syncthreads();
  const unsigned lanes = __ballot_sync(0xFFFFFFFFu, live);  // live lanes of this warp
  int E = 0;
  if (live) {
    if (!init) {
      const RoundKeys rk = make_round_keys(R.seed);
      const float beta_f = __double2float_rn(R.beta_next);
      const float bc = __fmul_rn(beta_f, GAUSS_LOG2E_SCALED);
      const int theta = R.theta_next;
      const uint32_t T0 = (uint32_t)R.sweeps;
#pragma unroll 1
      for (int t = 0; t < theta; ++t) {
        half_sweep_gauss1d<TPB, 0>(col, s_J, N, WR, nl, (uint32_t)slot, T0 + (uint32_t)t, rk, beta_f, bc, lanes,
                                   R.one);
        half_sweep_gauss1d<TPB, 1>(col, s_J, N, WR, nl, (uint32_t)slot, T0 + (uint32_t)t, rk, beta_f, bc, lanes,
                                   R.one);
      }
    }
    E = energy_gauss1d<TPB>(col, s_J, WR, nl, R.gC0);
    uint4* d4 = reinterpret_cast<uint4*>(R.spins[nxt] + (size_t)slot * W);
    for (int q = 0; q < W / 4; ++q) {
      uint4 v;
      v.x = (4 * q + 0 < WR) ? col[(4 * q + 0) * TPB] : 0u;
      v.y = (4 * q + 1 < WR) ? col[(4 * q + 1) * TPB] : 0u;
      v.z = (4 * q + 2 < WR) ? col[(4 * q + 2) * TPB] : 0u;
      v.w = (4 * q + 3 < WR) ? col[(4 * q + 3) * TPB] : 0u;
      d4[q] = v;
    }
  }
  measure_store_gauss1d(R, nxt, slot, live, E);
}

template <int TPB>
static cudaError_t launch_g1d_t(RunDev* runs, const Work* table, int nwork, int WR, cudaStream_t st, bool init) {
  const size_t sm = sizeof(uint32_t) * (32 * (size_t)WR + (size_t)WR * TPB);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_gauss1d<TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (nwork <= 0) return cudaSuccess;
  k_sweep_gauss1d<TPB><<<nwork, TPB, sm, st>>>(runs, table, init ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_gauss1d(int tpb, RunDev* runs, const Work* table, int nwork, int WR, cudaStream_t st, bool init) {
  switch (tpb) {
    case 32: return launch_g1d_t<32>(runs, table, nwork, WR, st, init);
    case 64: return launch_g1d_t<64>(runs, table, nwork, WR, st, init);
    case 128: return launch_g1d_t<128>(runs, table, nwork, WR, st, init);
    case 256: return launch_g1d_t<256>(runs, table, nwork, WR, st, init);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pa
