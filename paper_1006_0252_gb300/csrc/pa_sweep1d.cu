// pa_sweep1d.cu -- fused replica copy + checkerboard Metropolis sweeps +
// energy measurement for +-1 / diluted chains (Sec. 4: the 1D spin glass).
//
// Bit p of word w of a replica is site 32 w + p; colour = site parity.  A
// bond may be absent (J = 0, e.g. the wrap bond of an open chain), so the
// per-site energy change is dE = 4 n - 2 z_i with n satisfied bonds of the z_i
// present ones: n = 2 (dE = 4) and z_i = 1, n = 1 (dE = 2) are the rises that
// draw on the uniform.
#include "pa_lattice3d.cuh"

namespace pa {

// Bond masks of one chain run: [4][W] words: JP (coupling i->i+1 is -1),
// JM (coupling i-1->i is -1), PP (bond i->i+1 present), PM (bond i-1->i present).
enum { C_JP = 0, C_JM = 1, C_PP = 2, C_PM = 3 };

__device__ __forceinline__ uint32_t chain_valid(int w, int WR, int nl) {
  return (w + 1 < WR || nl == 32) ? 0xFFFFFFFFu : ((1u << nl) - 1u);
}

// Satisfied present bonds (i, i+1) of words w0 .. w1-1 of the column.
__device__ __forceinline__ int satisfied1d(const uint32_t* __restrict__ col, int CS, const uint32_t* __restrict__ s_bond,
                                           int W, int WR, int nl, int w0, int w1) {
  const uint32_t first = col[0];
  int sat = 0;
  for (int w = w0; w < w1; ++w) {
    const uint32_t curw = col[w * CS];
    const uint32_t nbp = (w + 1 < WR) ? __funnelshift_r(curw, col[(w + 1) * CS], 1)
                                      : ((curw >> 1) | ((first & 1u) << (nl - 1)));
    sat += __popc((curw ^ nbp ^ s_bond[C_JP * W + w]) & s_bond[C_PP * W + w]);
  }
  return sat;
}

// Compare chain (see lt_mask in pa_sweep3d.cuh): bit 2m of the result is
// [u_m < thr] for the 16 colour-c sites of a chain word.
__device__ __forceinline__ uint32_t lt_mask16(const uint32_t (&u)[16], uint32_t thr) {
  uint32_t ge = 0u;
#pragma unroll
  for (int m = 15; m >= 0; --m)
    asm("{\n\t.reg .u32 t;\n\tsub.cc.u32 t, %1, %2;\n\taddc.u32 %0, %3, %3;\n\t}"
        : "=r"(ge)
        : "r"(u[m]), "r"(thr), "r"(ge));
  uint32_t x = ~ge & 0xFFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

// Minimum of the 16 uniforms of a word (a tree of two-input minima).
__device__ __forceinline__ uint32_t min16(const uint32_t (&u)[16]) {
  uint32_t m[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) m[i] = min(u[i], u[i + 8]);
#pragma unroll
  for (int i = 0; i < 4; ++i) m[i] = min(m[i], m[i + 4]);
  return min(min(m[0], m[2]), min(m[1], m[3]));
}

// Words w0 .. w1-1 of one replica (a column, word w at col[w * CS]), colour
// c.  Colour-c sites read only colour-(1-c) neighbours, so the word ranges of
// the P threads of a replica are swept at once; the neighbour words outside
// the range (w0 - 1, w1, the wrap words) only contribute colour-(1-c) bits.
// The uniforms of word w are calls 4w .. 4w+3 of the colour: half-sweep
// entries at half[4w + k] (half already offset for this thread's range).
// Compares: dE = 2 arises only at sites with one bond present (a chain's ends
// and absent bonds), so thr(dE=2) is compared only in words holding such a
// site; thr(dE=4) in every word, except that at low temperature (thr4 <
// 2^22) a word whose uniforms' minimum is not below thr4 in any lane of the
// warp skips it (then no rise is accepted).
// Every thread of a replica runs WPP iterations, whatever its range holds (the
// last range may be short or empty), so that the warp votes below are taken
// by all live lanes together; an iteration past the range reads and writes
// nothing and votes with no compare results.
__device__ __forceinline__ void half_sweep1d(uint32_t* __restrict__ col, int CS, const uint32_t* __restrict__ s_bond,
                                             int W, int WR, int nl, int w0, int w1, int WPP, uint32_t c,
                                             const uint4* __restrict__ half, const SweepKey& key, const RoundKeys& rk,
                                             uint32_t T2, uint32_t T4, unsigned lanes) {
  const uint32_t first = col[0];
  const uint32_t last = col[(WR - 1) * CS];
  uint32_t prev = (w0 > 0 && w0 < WR) ? col[(w0 - 1) * CS] : last;
  uint32_t curw = (w0 < WR) ? col[w0 * CS] : 0u;
#pragma unroll 1
  for (int i = 0; i < WPP; ++i) {
    const int w = w0 + i;
    const bool act = w < w1;
    uint32_t nextw = 0u, need4 = 0u, need2 = 0u, e2 = 0u, e4 = 0u;
    uint32_t u[16];
    if (act) {
      nextw = (w + 1 < WR) ? col[(w + 1) * CS] : first;
      const uint32_t nbp = (w + 1 < WR) ? __funnelshift_r(curw, nextw, 1)
                                        : ((curw >> 1) | ((first & 1u) << (nl - 1)));
      const uint32_t nbm = (w > 0) ? __funnelshift_l(prev, curw, 1) : ((curw << 1) | ((last >> (nl - 1)) & 1u));
      const uint32_t pp = s_bond[C_PP * W + w], pm = s_bond[C_PM * W + w];
      const uint32_t bp = (curw ^ nbp ^ s_bond[C_JP * W + w]) & pp;
      const uint32_t bm = (curw ^ nbm ^ s_bond[C_JM * W + w]) & pm;
      need4 = bp & bm;
      need2 = (bp ^ bm) & (pp ^ pm);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const u32x4 v = philox_sweep(half[4 * w + q], key, rk);
        u[4 * q + 0] = v.a;
        u[4 * q + 1] = v.b;
        u[4 * q + 2] = v.c;
        u[4 * q + 3] = v.d;
      }
      if ((((pp ^ pm) >> c) & 0x55555555u) != 0u) e2 = lt_mask16(u, T2);
    }
    if (T4 < (1u << 22)) {
      if (__any_sync(lanes, act && min16(u) < T4) && act) e4 = lt_mask16(u, T4);
    } else if (act) {
      e4 = lt_mask16(u, T4);
    }
    if (act) {
      const uint32_t cm = (0x55555555u << c) & chain_valid(w, WR, nl);
      const uint32_t acc = cm & ~(need4 & ~(e4 << c)) & ~(need2 & ~(e2 << c));
      const uint32_t nw = curw ^ acc;
      col[w * CS] = nw;
      prev = nw;
      curw = nextw;
    }
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

// Shape of a chain sweep block: NR = TPB / P replicas, P threads per replica
// on ranges of WPP = ceil(WR / P) words; S = 4 WPP calls per range (the
// padding stride of the half-sweep table); CS the column stride that puts the
// P threads of a replica on different banks.
struct Chain1dShape {
  int NR, WPP, S, CS, Q, HB, NH;
};

__host__ __device__ inline Chain1dShape chain1d_shape(int TPB, int P, int WR) {
  Chain1dShape sh;
  sh.NR = TPB / P;
  sh.WPP = (WR + P - 1) / P;
  sh.Q = 4 * WR;
  sh.S = P == 1 ? sh.Q : 4 * sh.WPP;
  sh.HB = sh.Q + sh.Q / sh.S + 1;
  sh.CS = sh.NR;
  for (int cs = sh.NR; cs < sh.NR + 32 && P > 1; ++cs) {
    const int m = (sh.WPP * cs) % 32;
    if (m % (32 / P) == 0 && ((m / (32 / P)) & 1)) {
      sh.CS = cs;
      break;
    }
  }
  // half-sweep tables held at once (as for the cubic kernels): with one
  // thread per replica even, 2 .. 20, in about 216 bytes per thread with the
  // other tables; with several, two, double-buffered
  const int W = (WR + 3) / 4 * 4;  // words of a replica with padding; bonds [4][W]
  const int room = 216 * TPB - 4 * (4 * W + WR * sh.CS);
  const int nh = room > 0 ? room / (16 * sh.HB) : 0;
  sh.NH = P > 1 ? 2 : (nh >= 20 ? 20 : (nh < 2 ? 2 : (nh & ~1)));
  return sh;
}

__host__ __device__ inline size_t chain1d_smem_words(const Chain1dShape& sh, int W, int WR) {
  return 4 * (size_t)sh.NH * sh.HB + 4 * (size_t)W + (size_t)WR * sh.CS;
}

// Sec. 2 for chains: gather of the resampled population, theta checkerboard
// sweeps at beta', energy; block b takes work item b / P (TPB slots of one
// run) and its (b mod P)-th share of TPB / P replicas.
template <int TPB, int P>
__global__ void __launch_bounds__(TPB) k_sweep1d(RunDev* __restrict__ runs, const Work* __restrict__ table) {
  extern __shared__ __align__(16) uint32_t smem[];
  constexpr int RW = 32 / P;
  const Work wk = table[blockIdx.x / P];
  RunDev& R = runs[wk.run];
  if (R.skip) return;
  const int64_t Rn = R.R_next;
  const int W = R.W, WR = R.Wr, nl = R.N - 32 * (R.Wr - 1);
  const Chain1dShape sh = chain1d_shape(TPB, P, WR);
  const int64_t first = (int64_t)wk.first + (int64_t)(blockIdx.x % P) * sh.NR;
  if (first >= Rn) return;
  uint4* s_tab = reinterpret_cast<uint4*>(smem);
  uint32_t* s_bond = smem + 4 * sh.NH * sh.HB;
  uint32_t* s_spin = s_bond + 4 * W;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < 4 * W; i += TPB) s_bond[i] = R.bonds[i];
  const RoundKeys rk = make_round_keys(R.seed);
  const int r = (tid >> 5) * RW + (lane % RW);
  const int part = lane / RW;
  const int64_t slot = first + r;
  const bool live = slot < Rn;
  const int cur = R.cur, nxt = cur ^ 1;
  const int CS = sh.CS;
  uint32_t* col = s_spin + r;
  if (live) {
    const int32_t src = R.src[slot];
    const uint4* p4 = reinterpret_cast<const uint4*>(R.spins[cur] + (size_t)src * W);
    for (int q = part; q < W / 4; q += P) {
      const uint4 v = p4[q];
      if (4 * q + 0 < WR) col[(4 * q + 0) * CS] = v.x;
      if (4 * q + 1 < WR) col[(4 * q + 1) * CS] = v.y;
      if (4 * q + 2 < WR) col[(4 * q + 2) * CS] = v.z;
      if (4 * q + 3 < WR) col[(4 * q + 3) * CS] = v.w;
    }
  }
  __syncthreads();
  const unsigned lanes = __ballot_sync(0xFFFFFFFFu, live);  // live lanes of this warp
  const uint32_t T2 = R.thr[1], T4 = R.thr[2];
  const int theta = R.theta_next;
  const uint32_t T0 = (uint32_t)R.sweeps;
  const int w0 = min(part * sh.WPP, WR), w1 = min(w0 + sh.WPP, WR);
  if (P > 1) {
    // several threads per replica: one table per half sweep, double-buffered,
    // behind a block barrier that also orders the word ranges' half sweeps;
    // every thread of the block passes the barriers
#pragma unroll 1
    for (int t = 0; t < theta; ++t) {
      const uint32_t T = T0 + (uint32_t)t;
      const SweepKey key = sweep_key((uint32_t)slot, T, rk);
      const uint32_t A1 = PHILOX_MUL1 * T;
#pragma unroll 1
      for (uint32_t c = 0; c < 2; ++c) {
        uint4* half = s_tab + ((2 * t + (int)c) & 1) * sh.HB;
        for (int q = tid; q < sh.Q; q += TPB)
          half[q + q / sh.S] = sweep_half_entry(sweep_call_entry((uint32_t)q, TAG_SWEEP + c, rk), A1);
        __syncthreads();
        if (live) half_sweep1d(col, CS, s_bond, W, WR, nl, w0, w1, sh.WPP, c, half + part, key, rk, T2, T4, lanes);
      }
    }
  } else {
    // one thread per replica: half sweeps in chunks of NH tables, one block
    // barrier per chunk
    const int nhalf = 2 * theta;
    SweepKey key;
#pragma unroll 1
    for (int h0 = 0; h0 < nhalf; h0 += sh.NH) {
      if (h0 > 0) __syncthreads();  // the previous chunk's tables are no longer read
      const int nh = min(sh.NH, nhalf - h0);
      for (int i = tid; i < nh * sh.Q; i += TPB) {
        const int j = i / sh.Q, q = i - j * sh.Q;
        const int h = h0 + j;
        const uint32_t A1 = PHILOX_MUL1 * (T0 + (uint32_t)(h >> 1));
        s_tab[j * sh.HB + q + q / sh.S] =
            sweep_half_entry(sweep_call_entry((uint32_t)q, TAG_SWEEP + (uint32_t)(h & 1), rk), A1);
      }
      __syncthreads();
      if (live) {
#pragma unroll 1
        for (int j = 0; j < nh; ++j) {
          const uint32_t c = (uint32_t)j & 1u;  // h0 is even
          if (c == 0) key = sweep_key((uint32_t)slot, T0 + (uint32_t)((h0 + j) >> 1), rk);
          half_sweep1d(col, CS, s_bond, W, WR, nl, w0, w1, sh.WPP, c, s_tab + j * sh.HB, key, rk, T2,
                       T4, lanes);
        }
      }
    }
  }
  __syncthreads();  // every word range swept before the energy reads its neighbour words
  int E = 0;
  if (live) {
    int sat = satisfied1d(col, CS, s_bond, W, WR, nl, w0, w1);
#pragma unroll
    for (int off = RW; off < 32; off <<= 1) sat += __shfl_xor_sync(lanes, sat, off);
    E = R.Nb - 2 * sat;
    uint4* d4 = reinterpret_cast<uint4*>(R.spins[nxt] + (size_t)slot * W);
    for (int q = part; q < W / 4; q += P) {
      uint4 v;
      v.x = (4 * q + 0 < WR) ? col[(4 * q + 0) * CS] : 0u;
      v.y = (4 * q + 1 < WR) ? col[(4 * q + 1) * CS] : 0u;
      v.z = (4 * q + 2 < WR) ? col[(4 * q + 2) * CS] : 0u;
      v.w = (4 * q + 3 < WR) ? col[(4 * q + 3) * CS] : 0u;
      d4[q] = v;
    }
  }
  measure_store1d(R, nxt, slot, live && part == 0, E);
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
    E = R.Nb - 2 * satisfied1d(col, TPB, s_bond, W, WR, nl, 0, WR);
    store_column1d<TPB>(R.spins[0] + (size_t)slot * W, col, W, WR);
  }
  measure_store1d(R, 0, slot, live, E);
}

template <int TPB, int P>
static cudaError_t launch_sweep1d_p(RunDev* runs, const Work* table, int nwork, int W, int WR, cudaStream_t st) {
  if constexpr (TPB / P < 4 || (P > 1 && TPB < 64)) {
    return cudaErrorInvalidValue;
  } else {
    const Chain1dShape sh = chain1d_shape(TPB, P, WR);
    const size_t sm = sizeof(uint32_t) * chain1d_smem_words(sh, W, WR);
    if (sm > 48 * 1024) {
      cudaError_t e =
          cudaFuncSetAttribute(k_sweep1d<TPB, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    if (nwork <= 0) return cudaSuccess;
    k_sweep1d<TPB, P><<<nwork * P, TPB, sm, st>>>(runs, table);
    return cudaGetLastError();
  }
}

template <int TPB>
static cudaError_t launch1d_t(RunDev* runs, const Work* table, int nwork, int W, int WR, cudaStream_t st, bool init,
                              int split) {
  if (!init) {
    switch (split) {
      case 1: return launch_sweep1d_p<TPB, 1>(runs, table, nwork, W, WR, st);
      case 2: return launch_sweep1d_p<TPB, 2>(runs, table, nwork, W, WR, st);
      case 4: return launch_sweep1d_p<TPB, 4>(runs, table, nwork, W, WR, st);
      case 8: return launch_sweep1d_p<TPB, 8>(runs, table, nwork, W, WR, st);
      default: return cudaErrorInvalidValue;
    }
  }
  const size_t sm = sizeof(uint32_t) * (4 * (size_t)W + (size_t)WR * TPB);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_init1d<TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (nwork <= 0) return cudaSuccess;
  k_init1d<TPB><<<nwork, TPB, sm, st>>>(runs, table);
  return cudaGetLastError();
}

// Threads per replica for chains: 1, 2, 4 or 8 (word ranges of ceil(WR / P)).
bool sweep1d_split_ok(int split) { return split == 1 || split == 2 || split == 4 || split == 8; }

cudaError_t launch_sweep1d(int tpb, int split, RunDev* runs, const Work* table, int nwork, int W, int WR,
                           cudaStream_t st, bool init) {
  switch (tpb) {
    case 32: return launch1d_t<32>(runs, table, nwork, W, WR, st, init, split);
    case 64: return launch1d_t<64>(runs, table, nwork, W, WR, st, init, split);
    case 128: return launch1d_t<128>(runs, table, nwork, W, WR, st, init, split);
    case 256: return launch1d_t<256>(runs, table, nwork, W, WR, st, init, split);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pa
