// pa_gauss1d.cu -- fused replica copy + checkerboard Metropolis sweeps +
// energy measurement for chains with Gaussian couplings (Sec. 4: the periodic
// 1D spin glass the paper compares with exact transfer matrices).
//
// Bit p of word w of a replica is site 32 w + p; colour = site parity.  The
// couplings J_q[i] (bond i -> i+1, J_q[N-1] the wrap bond, 0 = absent) sit in
// shared memory as int32.  For site i with a+ = 1 where s_{i+1} != s_i and
// a- = 1 where s_{i-1} != s_i:
//   dE_i = 4 (a+ J[i] + a- J[i-1]) - 2 (J[i] + J[i-1]),
// one of four values per site.  Every block tabulates, once per launch (one
// beta), the integer acceptance threshold gauss_threshold(dE, beta) of the
// four patterns of every site (16 N bytes), so that a site's decision is one
// table load and one integer compare (u >> 8) < thr, which is the Metropolis
// decision of pa_gauss.cuh exactly.  The sweep uniforms come from the call
// and half-sweep tables of pa_lattice3d.cuh (the +-1 chain kernel's keying).
#include "pa_gauss.cuh"
#include "pa_lattice3d.cuh"

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

// Threshold table of a chain: [2 colours][WR words][16 ranks][4 patterns]
// (256 bytes per word and colour), pattern p = a+ | a- << 1 for the colour-c
// site i = 32 w + c + 2 m; sites past the chain's end get entries too (their
// flips are masked).
__device__ __forceinline__ uint32_t gchain_threshold(const int32_t* __restrict__ s_J, int N, int idx,
                                                     float beta_f) {
  const int p = idx & 3, m = (idx >> 2) & 15, cw = idx >> 6;
  const int c = cw & 1, w = cw >> 1;
  const int i = 32 * w + c + 2 * m;
  const int32_t jp = s_J[i];
  const int32_t jm = (i == 0) ? s_J[N - 1] : s_J[i - 1];
  const int32_t acc = ((p & 1) ? jp : 0) + ((p & 2) ? jm : 0);
  return gauss_threshold(4 * acc - 2 * (jp + jm), beta_f);
}

// Colour-c half sweep of one replica (a column, word w at col[w * TPB]):
// per word the anti-alignment bits, its 16 uniforms (calls 4w .. 4w+3 of the
// half-sweep table), then per site the table load and the compare.  The
// two pattern bits of the sites m = 4j + r sit in byte j of F[r] at bits
// 2-3, so one byte permute yields the entry's address (the word's
// 256-byte-aligned table in bytes 1-3, 4 p in byte 0, 16 m as the offset).
template <int TPB>
__device__ __forceinline__ void half_sweep_gtab1d(uint32_t* __restrict__ col, uint32_t thr_base, int WR, int nl,
                                                  uint32_t c, const uint4* __restrict__ half, const SweepKey& key,
                                                  const RoundKeys& rk, uint32_t one) {
  const uint32_t first = col[0];
  const uint32_t last = col[(WR - 1) * TPB];
  uint32_t prev = last, curw = first;
#pragma unroll 1
  for (int w = 0; w < WR; ++w) {
    const uint32_t nextw = (w + 1 < WR) ? col[(w + 1) * TPB] : first;
    const uint32_t nbp = (w + 1 < WR) ? __funnelshift_r(curw, nextw, 1)
                                      : ((curw >> 1) | ((first & 1u) << (nl - 1)));
    const uint32_t nbm = (w > 0) ? __funnelshift_l(prev, curw, 1)
                                 : ((curw << 1) | ((last >> (nl - 1)) & 1u));
    const uint32_t x = (((curw ^ nbp) >> c) & 0x55555555u) | ((((curw ^ nbm) >> c) & 0x55555555u) << 1);
    uint32_t F[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) F[r] = ((x >> (2 * r)) << 2) & 0x0C0C0C0Cu;
    uint32_t u[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const u32x4 v = philox_sweep(half[4 * w + q], key, rk);
      u[4 * q + 0] = v.a;
      u[4 * q + 1] = v.b;
      u[4 * q + 2] = v.c;
      u[4 * q + 3] = v.d;
    }
    const uint32_t base = thr_base + (uint32_t)(2 * w + (int)c) * 256u;
    uint32_t flip = 0u;
    static_for<0, 16>([&](auto mc) {
      constexpr int m = decltype(mc)::value;
      const uint32_t addr = __byte_perm(F[m & 3], base, (uint32_t)(m >> 2) | 0x7650u);
      uint32_t t;
      asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(t) : "r"(addr), "n"(m * 16));
      // the bit set by a predicated multiply-add on the multiply pipe (one == 1)
      asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %3, %4, %0;\n\t}"
          : "+r"(flip)
          : "r"(u[m] >> 8), "r"(t), "r"(one), "n"(1u << (2 * m)));
    });
    const uint32_t nw = curw ^ ((flip << c) & gchain_valid(w, WR, nl));
    col[w * TPB] = nw;
    prev = nw;
    curw = nextw;
  }
}

// Shared memory of the chain kernel (words): 64 of alignment slack, the
// threshold table (128 WR), the call entries (2 Q uint4, Q = 4 WR calls per
// colour), NH half-sweep tables (NH Q uint4), the couplings padded to whole
// words (32 WR) and the spin columns (WR TPB).  NH: even, 2 .. 20, in about
// 216 bytes per thread with the rest.
struct GChainShape {
  int Q, NH;
  size_t words;
};
__host__ __device__ inline GChainShape gchain_shape(int TPB, int WR) {
  GChainShape sh;
  sh.Q = 4 * WR;
  const int other = 4 * (64 + 128 * WR + 8 * sh.Q + 32 * WR + WR * TPB);
  const int room = 216 * TPB - other;
  const int nh = room > 0 ? room / (16 * sh.Q) : 0;
  sh.NH = nh >= 20 ? 20 : (nh < 2 ? 2 : (nh & ~1));
  sh.words = 64 + 128 * (size_t)WR + 8 * (size_t)sh.Q + 4 * (size_t)sh.NH * sh.Q + 32 * (size_t)WR +
             (size_t)WR * TPB;
  return sh;
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
  extern __shared__ __align__(16) uint32_t smem[];
  const Work wk = table[blockIdx.x];
  RunDev& R = runs[wk.run];
  if (!init && R.skip) return;
  const int64_t Rn = init ? R.R : R.R_next;
  if ((int64_t)wk.first >= Rn) return;
  const int N = R.N, W = R.W, WR = R.Wr, nl = N - 32 * (WR - 1);
  const GChainShape sh = gchain_shape(TPB, WR);
  const uint32_t smem_addr = (uint32_t)__cvta_generic_to_shared(smem);
  uint32_t* s_thr = smem + ((256u - (smem_addr & 255u)) & 255u) / 4u;  // 256-byte aligned
  uint4* s_tab = reinterpret_cast<uint4*>(s_thr + 128 * WR);           // calls, then half-sweep tables
  int32_t* s_J = reinterpret_cast<int32_t*>(s_thr + 128 * WR + 8 * sh.Q + 4 * sh.NH * sh.Q);
  uint32_t* s_spin = reinterpret_cast<uint32_t*>(s_J + 32 * WR);
  const int tid = threadIdx.x;
  for (int i = tid; i < 32 * WR; i += TPB) s_J[i] = (i < N) ? R.gJ[i] : 0;
  const RoundKeys rk = make_round_keys(R.seed);
  if (!init)
    for (int i = tid; i < 2 * sh.Q; i += TPB) {
      const int c = i / sh.Q, q = i - c * sh.Q;
      s_tab[i] = sweep_call_entry((uint32_t)q, TAG_SWEEP + (uint32_t)c, rk);
    }
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
  __syncthreads();  // couplings (and the call entries) in place
  if (!init) {
    const float beta_f = __double2float_rn(R.beta_next);
    for (int i = tid; i < 128 * WR; i += TPB) s_thr[i] = gchain_threshold(s_J, N, i, beta_f);
    const uint32_t thr_base = (uint32_t)__cvta_generic_to_shared(s_thr);
    const int theta = R.theta_next;
    const uint32_t T0 = (uint32_t)R.sweeps;
    const int nhalf = 2 * theta;
    SweepKey key;
    // half sweeps in chunks of NH tables behind one block barrier each; a
    // thread sweeps its own replica, so nothing else orders the half sweeps
#pragma unroll 1
    for (int h0 = 0; h0 < nhalf; h0 += sh.NH) {
      if (h0 > 0) __syncthreads();  // the previous chunk's tables are no longer read
      const int nh = min(sh.NH, nhalf - h0);
      for (int i = tid; i < nh * sh.Q; i += TPB) {
        const int j = i / sh.Q, q = i - j * sh.Q;
        const int h = h0 + j;
        const uint32_t A1 = PHILOX_MUL1 * (T0 + (uint32_t)(h >> 1));
        s_tab[2 * sh.Q + j * sh.Q + q] = sweep_half_entry(s_tab[(h & 1) * sh.Q + q], A1);
      }
      __syncthreads();  // the tables (and, first time, the thresholds) in place
      if (live) {
#pragma unroll 1
        for (int j = 0; j < nh; ++j) {
          const uint32_t c = (uint32_t)j & 1u;  // h0 is even
          if (c == 0) key = sweep_key((uint32_t)slot, T0 + (uint32_t)((h0 + j) >> 1), rk);
          half_sweep_gtab1d<TPB>(col, thr_base, WR, nl, c, s_tab + 2 * sh.Q + j * sh.Q, key, rk, R.one);
        }
      }
    }
  }
  int E = 0;
  if (live) {
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
  const size_t sm = sizeof(uint32_t) * gchain_shape(TPB, WR).words;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_gauss1d<TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (nwork <= 0) return cudaSuccess;
  k_sweep_gauss1d<TPB><<<nwork, TPB, sm, st>>>(runs, table, init ? 1 : 0);
  return cudaGetLastError();
}

size_t gauss1d_smem_bytes(int tpb, int WR) { return sizeof(uint32_t) * gchain_shape(tpb, WR).words; }

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
