// pa_sweep1d.cu -- fused replica copy + checkerboard Metropolis sweeps +
// energy measurement for +-1 / diluted chains (Sec. 4: the 1D spin glass).
//
// Bit p of word w of a replica is site 32 w + p; colour = site parity.  A
// bond may be absent (J = 0, e.g. the wrap bond of an open chain), so the
// per-site energy change is dE = 4 n - 2 z_i with n satisfied bonds of the z_i
// present ones: n = 2 (dE = 4) and z_i = 1, n = 1 (dE = 2) are the rises that
// draw on the uniform.
#include "pa_device.cuh"

namespace pa {

// Bond masks of one chain run: [4][W] words: JP (coupling i->i+1 is -1),
// JM (coupling i-1->i is -1), PP (bond i->i+1 present), PM (bond i-1->i present).
enum { C_JP = 0, C_JM = 1, C_PP = 2, C_PM = 3 };

__device__ __forceinline__ uint32_t chain_valid(int w, int WR, int nl) {
  return (w + 1 < WR || nl == 32) ? 0xFFFFFFFFu : ((1u << nl) - 1u);
}

template <int TPB>
__device__ __forceinline__ int energy1d(const uint32_t* __restrict__ col,
                                        const uint32_t* __restrict__ s_bond, int W, int WR, int nl,
                                        int Nb) {
  const uint32_t first = col[0];
  int sat = 0;
  uint32_t curw = first;
  for (int w = 0; w < WR; ++w) {
    uint32_t nbp;
    if (w + 1 < WR) {
      const uint32_t nextw = col[(w + 1) * TPB];
      nbp = __funnelshift_r(curw, nextw, 1);
      sat += __popc((curw ^ nbp ^ s_bond[C_JP * W + w]) & s_bond[C_PP * W + w]);
      curw = nextw;
    } else {
      nbp = (curw >> 1) | ((first & 1u) << (nl - 1));
      sat += __popc((curw ^ nbp ^ s_bond[C_JP * W + w]) & s_bond[C_PP * W + w]);
    }
  }
  return Nb - 2 * sat;
}

template <int TPB>
__device__ __forceinline__ void half_sweep1d(uint32_t* __restrict__ col,
                                             const uint32_t* __restrict__ s_bond, int W, int WR,
                                             int nl, uint32_t slot, uint32_t T, uint32_t c,
                                             const RoundKeys& rk, uint32_t T2, uint32_t T4,
                                             unsigned lanes) {
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
    const uint32_t pp = s_bond[C_PP * W + w], pm = s_bond[C_PM * W + w];
    const uint32_t bp = (curw ^ nbp ^ s_bond[C_JP * W + w]) & pp;
    const uint32_t bm = (curw ^ nbm ^ s_bond[C_JM * W + w]) & pm;
    const uint32_t need4 = bp & bm;
    const uint32_t need2 = (bp ^ bm) & (pp ^ pm);
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
    // thr(dE=2) >= thr(dE=4): the second compare is needed only where the
    // first succeeds; skipped for the word when no lane of the warp needs it
    uint32_t e2 = 0u, e4 = 0u;
#pragma unroll
    for (int m = 0; m < 16; ++m) e2 |= (u[m] < T2) ? (1u << (2 * m)) : 0u;
    if (__any_sync(lanes, e2 != 0u)) {
#pragma unroll
      for (int m = 0; m < 16; ++m) e4 |= (u[m] < T4) ? (1u << (2 * m)) : 0u;
    }
    const uint32_t cm = (0x55555555u << c) & chain_valid(w, WR, nl);
    const uint32_t acc = cm & ~(need4 & ~(e4 << c)) & ~(need2 & ~(e2 << c));
    const uint32_t nw = curw ^ acc;
    col[w * TPB] = nw;
    prev = nw;
    curw = nextw;
  }
}

__device__ __forceinline__ void measure_store1d(RunDev& R, int nxt, int64_t slot, bool live, int E) {
  if (live) {
    R.E[nxt][slot] = E;
    atomicAdd(&R.hist[nxt][(E + R.Nb) >> 1], 1u);
  }
  long long e = live ? (long long)E : 0ll;
  long long e2 = e * e;
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) {
    e += __shfl_xor_sync(0xFFFFFFFFu, e, sh);
    e2 += __shfl_xor_sync(0xFFFFFFFFu, e2, sh);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&R.sumE_next, (unsigned long long)e);
    atomicAdd(&R.sumE2_next, (unsigned long long)e2);
  }
}

template <int TPB>
__device__ __forceinline__ void store_column1d(uint32_t* __restrict__ dst,
                                               const uint32_t* __restrict__ col, int W, int WR) {
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  for (int q = 0; q < W / 4; ++q) {
    uint4 v;
    v.x = (4 * q + 0 < WR) ? col[(4 * q + 0) * TPB] : 0u;
    v.y = (4 * q + 1 < WR) ? col[(4 * q + 1) * TPB] : 0u;
    v.z = (4 * q + 2 < WR) ? col[(4 * q + 2) * TPB] : 0u;
    v.w = (4 * q + 3 < WR) ? col[(4 * q + 3) * TPB] : 0u;
    d4[q] = v;
  }
}

template <int TPB>
__global__ void __launch_bounds__(TPB) k_sweep1d(RunDev* __restrict__ runs,
                                                 const Work* __restrict__ table) {
  extern __shared__ uint32_t smem[];
  const Work wk = table[blockIdx.x];
  RunDev& R = runs[wk.run];
  if (R.skip) return;
  const int64_t Rn = R.R_next;
  if ((int64_t)wk.first >= Rn) return;
  const int W = R.W, WR = R.Wr, nl = R.N - 32 * (R.Wr - 1);
  uint32_t* s_bond = smem;
  uint32_t* s_spin = smem + 4 * W;
  const int tid = threadIdx.x;
  for (int i = tid; i < 4 * W; i += TPB) s_bond[i] = R.bonds[i];
  const int64_t slot = (int64_t)wk.first + tid;
  const bool live = slot < Rn;
  const int cur = R.cur, nxt = cur ^ 1;
  uint32_t* col = s_spin + tid;
  if (live) {
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
  __syncthreads();
  const unsigned lanes = __ballot_sync(0xFFFFFFFFu, live);  // live lanes of this warp
  int E = 0;
  if (live) {
    const RoundKeys rk = make_round_keys(R.seed);
    const uint32_t T2 = R.thr[1], T4 = R.thr[2];
    const int theta = R.theta_next;
    const uint32_t T0 = (uint32_t)R.sweeps;
#pragma unroll 1
    for (int t = 0; t < theta; ++t) {
#pragma unroll 1
      for (uint32_t c = 0; c < 2; ++c)
        half_sweep1d<TPB>(col, s_bond, W, WR, nl, (uint32_t)slot, T0 + (uint32_t)t, c, rk, T2, T4, lanes);
    }
    E = energy1d<TPB>(col, s_bond, W, WR, nl, R.Nb);
    store_column1d<TPB>(R.spins[nxt] + (size_t)slot * W, col, W, WR);
  }
  measure_store1d(R, nxt, slot, live, E);
}

template <int TPB>
__global__ void __launch_bounds__(TPB) k_init1d(RunDev* __restrict__ runs,
                                                const Work* __restrict__ table) {
  extern __shared__ uint32_t smem[];
  const Work wk = table[blockIdx.x];
  RunDev& R = runs[wk.run];
  const int64_t R0 = R.R;
  if ((int64_t)wk.first >= R0) return;
  const int W = R.W, WR = R.Wr, nl = R.N - 32 * (R.Wr - 1);
  uint32_t* s_bond = smem;
  uint32_t* s_spin = smem + 4 * W;
  const int tid = threadIdx.x;
  for (int i = tid; i < 4 * W; i += TPB) s_bond[i] = R.bonds[i];
  const int64_t slot = (int64_t)wk.first + tid;
  const bool live = slot < R0;
  uint32_t* col = s_spin + tid;
  if (live) {
    for (int w4 = 0; w4 < W / 4; ++w4) {
      const u32x4 u = philox_seeded(R.seed, (uint32_t)w4, (uint32_t)slot, 0u, TAG_INIT);
      const uint32_t v[4] = {u.a, u.b, u.c, u.d};
      for (int i = 0; i < 4; ++i) {
        const int w = 4 * w4 + i;
        if (w < WR) col[w * TPB] = v[i] & chain_valid(w, WR, nl);
      }
    }
  }
  __syncthreads();
  int E = 0;
  if (live) {
    E = energy1d<TPB>(col, s_bond, W, WR, nl, R.Nb);
    store_column1d<TPB>(R.spins[0] + (size_t)slot * W, col, W, WR);
  }
  measure_store1d(R, 0, slot, live, E);
}

template <int TPB>
static cudaError_t launch1d_t(RunDev* runs, const Work* table, int nwork, int W, int WR,
                              cudaStream_t st, bool init) {
  const size_t sm = sizeof(uint32_t) * (4 * (size_t)W + (size_t)WR * TPB);
  auto kern = init ? k_init1d<TPB> : k_sweep1d<TPB>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (nwork <= 0) return cudaSuccess;
  kern<<<nwork, TPB, sm, st>>>(runs, table);
  return cudaGetLastError();
}

cudaError_t launch_sweep1d(int tpb, RunDev* runs, const Work* table, int nwork, int W, int WR,
                           cudaStream_t st, bool init) {
  switch (tpb) {
    case 32: return launch1d_t<32>(runs, table, nwork, W, WR, st, init);
    case 64: return launch1d_t<64>(runs, table, nwork, W, WR, st, init);
    case 128: return launch1d_t<128>(runs, table, nwork, W, WR, st, init);
    case 256: return launch1d_t<256>(runs, table, nwork, W, WR, st, init);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pa
