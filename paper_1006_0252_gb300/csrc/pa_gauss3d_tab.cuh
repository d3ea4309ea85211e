// pa_gauss3d_tab.cuh -- the Gaussian sweep (Sec. 4 couplings, Sec. 2 sweeps)
// with per-site acceptance thresholds, for edges L <= 8 and large blocks.
//
// A colour-c site i has six neighbours; with x_d = 1 where neighbour d is
// anti-aligned with s_i, its energy change is dE_i(x) = 4 sum_{d: x_d = 1}
// J_d - 2 S_i, one of 64 values fixed by the couplings.  At a given beta the
// Metropolis decision of pa_gauss.cuh (accept iff dE <= 0 or
// float(u >> 8) < lim(dE), lim = fexp(x) 2^24, every operation rounded as
// specified) compares the integer u >> 8 < 2^24 with a float lim in
// [0, 2^24], so it is exactly the integer compare (u >> 8) < thr with
//   thr = 2^24 (dE <= 0),  thr = ceil(lim(dE)) (dE > 0).
// At the start of a launch (one beta) every block tabulates thr for all 64
// patterns of every site of both colours in shared memory (L = 8: 2 x 16
// words x 16 sites x 64 x 4 B = 128 KB), computed with the decision's own
// arithmetic; a site's update is then its pattern, one table load and one
// integer compare: no energy sum, no exponential and no estimate window in
// the sweep.  Everything else (layout, window, keying, uniforms, P threads
// per replica, chunked half-sweep tables) is the cubic kernels'.
#pragma once
#include "pa_gauss3d.cuh"

namespace pa {

// Threshold table words: [2 colours][WR words][SITES ranks][64 patterns].
template <class GEO>
__host__ __device__ constexpr int gtab_words() {
  return 2 * GEO::WR * (GEO::K * GEO::L / 2) * 64;
}

// thr for pattern p of the colour-c site of rank m of word w: bit d of p is
// x_d (d = +x, -x, +y, -y, +z, -z as in gword3d).
template <class GEO>
__device__ __forceinline__ uint32_t gtab_entry(const int32_t* __restrict__ gJ, const int32_t* __restrict__ gS,
                                               int c, int w, int m, int p, float beta_f) {
  constexpr int WR = GEO::WR, SP = ((GEO::K * GEO::L / 2) + 3) & ~3;
  const int32_t* Jw = gJ + (c * 6 * WR + w) * SP + m;
  int32_t acc = 0;
#pragma unroll
  for (int d = 0; d < 6; ++d)
    if ((p >> d) & 1) acc += __ldg(Jw + d * WR * SP);
  return gauss_threshold(4 * acc - 2 * __ldg(gS + (c * WR + w) * SP + m), beta_f);
}

// flip |= 2^BIT where x < t: the compare on the integer ALU pipe, the bit set
// by a predicated multiply-add (2^BIT * one + flip, one == 1 at run time) on
// the multiply pipe, which the sweep leaves less busy (measured 6-7 % faster
// than setting the bit with integer logic).
template <int BIT>
__device__ __forceinline__ void set_bit_if_below(uint32_t& flip, uint32_t x, uint32_t t, uint32_t one) {
  asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %3, %4, %0;\n\t}"
      : "+r"(flip)
      : "r"(x), "r"(t), "r"(one), "n"(1u << BIT));
}

// Word g of row y: anti-alignment bits, the word's uniforms, then per site
// the table load at its pattern and the compare.  The pattern bits are
// gathered four sites to a register (sites m = 4j + r in byte j of F[r], x_d
// at bit d + 2 of the byte), so that one byte permute yields the table
// address: the site table's 256-byte-aligned base in bytes 1-3, 4 p in byte 0.
template <class GEO, int A>
__device__ __forceinline__ void tword3d(int g, int y, uint32_t s_thr, uint32_t (&rowm)[GEO::G],
                                        uint32_t (&row)[GEO::G], const uint32_t (&rowp)[GEO::G],
                                        const GaussHalf& gh, const RoundKeys& rk, uint32_t (&carry)[4]) {
  constexpr int G = GEO::G, L = GEO::L, K = GEO::K, WR = GEO::WR;
  constexpr int SITES = K * L / 2;
  const int w = y * G + g;
  const uint32_t s = row[g];
  const uint32_t c = gh.c;
  const uint32_t par0 = (c + (uint32_t)y + (uint32_t)g) & 1u;
  const uint32_t zp = (g + 1 < G) ? row[(g + 1) % G] : lanes_down<GEO>(row[0]);
  const uint32_t zm = (g > 0) ? row[(g + G - 1) % G] : lanes_up<GEO>(row[G - 1]);
  // pairs of directions at bits 2m (d even) and 2m + 1 (d odd)
  const uint32_t x01 = from_colour_positions<GEO>(s ^ rot_xp<GEO>(s), par0) |
                       (from_colour_positions<GEO>(s ^ rot_xm<GEO>(s), par0) << 1);
  const uint32_t x23 = from_colour_positions<GEO>(s ^ rowp[g], par0) |
                       (from_colour_positions<GEO>(s ^ rowm[g], par0) << 1);
  const uint32_t x45 = from_colour_positions<GEO>(s ^ zp, par0) | (from_colour_positions<GEO>(s ^ zm, par0) << 1);
  // F[r], byte j: site m = 4j + r (bits 2m, 2m+1 of x01 / x23 / x45 moved to
  // bits 2-3 / 4-5 / 6-7 of the byte)
  uint32_t F[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    F[r] = (((x01 >> (2 * r)) << 2) & 0x0C0C0C0Cu) | (((x23 >> (2 * r)) << 4) & 0x30303030u) |
           (((x45 >> (2 * r)) << 6) & 0xC0C0C0C0u);
  }
  const uint32_t r0 = (uint32_t)(w * SITES);  // colour-c rank of the word's first site
  uint32_t u[4 * word_calls<SITES, A>()];
  word_uniforms<SITES, A>(r0 >> 2, gh.half, gh.key, rk, carry, u);
  const uint32_t base = s_thr + (uint32_t)((c * WR + w) * SITES) * 256u;
  uint32_t flip = 0u;
  static_for<0, SITES>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    const uint32_t addr = __byte_perm(F[m & 3], base, (uint32_t)(m >> 2) | 0x7650u);
    uint32_t t;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(t) : "r"(addr), "n"(m * 256));
    set_bit_if_below<2 * m>(flip, u[A + m] >> 8, t, gh.one);
  });
  row[g] = s ^ to_colour_positions<GEO>(flip, par0);
}

template <class GEO, int CS, int YP>
__device__ __forceinline__ void trow3d(uint32_t* __restrict__ col, uint32_t s_thr, int y, uint32_t (&rowm)[GEO::G],
                                       uint32_t (&row)[GEO::G], uint32_t (&rowp)[GEO::G], const GaussHalf& gh,
                                       const RoundKeys& rk, uint32_t (&carry)[4]) {
  constexpr int G = GEO::G, L = GEO::L, K = GEO::K;
  constexpr int SITES = K * L / 2;
  const int yn = (y + 1 == L) ? 0 : y + 1;
#pragma unroll
  for (int g = 0; g < G; ++g) rowp[g] = col[(yn * G + g) * CS];
  if constexpr (SITES % 4 == 0) {
#pragma unroll
    for (int g = 0; g < G; ++g) tword3d<GEO, 0>(g, y, s_thr, rowm, row, rowp, gh, rk, carry);
  } else {
    static_for<0, G>([&](auto gc) {
      constexpr int g = decltype(gc)::value;
      constexpr int A = (SITES * (YP * G + g)) % 4;
      tword3d<GEO, A>(g, y, s_thr, rowm, row, rowp, gh, rk, carry);
    });
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    col[(y * G + g) * CS] = row[g];
    rowm[g] = row[g];
    row[g] = rowp[g];
  }
}

// One half sweep over rows y0 .. y0 + RPP - 1 (pairs of rows when the
// colour-c sites per word are not a multiple of 4), as half_sweep_gauss3d.
template <class GEO, int CS, int RPP>
__device__ __forceinline__ void half_sweep_gtab3d(uint32_t* __restrict__ col, uint32_t s_thr, const GaussHalf& gh,
                                                  const RoundKeys& rk, int y0) {
  constexpr int G = GEO::G, L = GEO::L, K = GEO::K;
  constexpr int SITES = K * L / 2;
  uint32_t rowm[G], row[G], rowp[G];
  uint32_t carry[4] = {0u, 0u, 0u, 0u};
  const int ym = (y0 == 0) ? L - 1 : y0 - 1;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    rowm[g] = col[(ym * G + g) * CS];
    row[g] = col[(y0 * G + g) * CS];
  }
  if constexpr (SITES % 4 == 0) {
#pragma unroll 1
    for (int i = 0; i < RPP; ++i) trow3d<GEO, CS, 0>(col, s_thr, y0 + i, rowm, row, rowp, gh, rk, carry);
  } else {
    static_assert(RPP % 2 == 0, "rows come in pairs");
#pragma unroll 1
    for (int i = 0; i < RPP; i += 2) {
      trow3d<GEO, CS, 0>(col, s_thr, y0 + i, rowm, row, rowp, gh, rk, carry);
      trow3d<GEO, CS, 1>(col, s_thr, y0 + i + 1, rowm, row, rowp, gh, rk, carry);
    }
  }
}

template <int L, int TPB, int P>
struct GTabShape {
  using GEO = Geo3<L>;
  static constexpr int NR = TPB / P;
  static constexpr int RPP = L / P;
  static constexpr int CS = split_stride(NR, RPP * GEO::G, P, TPB);
  static constexpr int NH = half_tables<GEO, TPB, P>(4 * (gtab_words<GEO>() + GEO::WR * CS));
  // + 64 words: the table starts at the first 256-byte boundary of the block's
  // shared memory
  static constexpr size_t SMEM_WORDS =
      64 + (size_t)gtab_words<GEO>() + sweep_table_words<GEO, P>(NH) + GEO::WR * CS;
};

// Sec. 2 with the Gaussian couplings of Sec. 4 (the decision of k_sweep_gauss3d
// through the threshold tables): gather of the resampled population, theta
// checkerboard sweeps at beta', the energy of every replica.  Block b takes
// work item b / P (TPB slots of one run) and its (b mod P)-th share.
template <int L, int TPB, int P>
__global__ void __launch_bounds__(TPB) k_sweep_gtab3d(RunDev* __restrict__ runs, const Work* __restrict__ table) {
  using GEO = Geo3<L>;
  using SH = GTabShape<L, TPB, P>;
  constexpr int WR = GEO::WR, W = GEO::W, SITES = GEO::K * L / 2;
  constexpr int RW = 32 / P, RPP = SH::RPP, CS = SH::CS;
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t smem_addr = (uint32_t)__cvta_generic_to_shared(smem);
  uint32_t* s_thr = smem + ((256u - (smem_addr & 255u)) & 255u) / 4u;                // gtab_words, 256-B aligned
  uint4* s_tab = reinterpret_cast<uint4*>(s_thr + gtab_words<GEO>());                // sweep_table_words
  uint32_t* s_spin = s_thr + gtab_words<GEO>() + sweep_table_words<GEO, P>(SH::NH);  // [WR][CS]
  const Work wk = table[blockIdx.x / P];
  RunDev& R = runs[wk.run];
  if (R.skip) return;
  const int64_t Rn = R.R_next;
  const int64_t first = (int64_t)wk.first + (int64_t)(blockIdx.x % P) * SH::NR;
  if (first >= Rn) return;
  const int tid = threadIdx.x, lane = tid & 31;
  const float beta_f = __double2float_rn(R.beta_next);
  for (int i = tid; i < gtab_words<GEO>(); i += TPB) {
    const int p = i & 63, site = i >> 6;  // site = (c * WR + w) * SITES + m
    const int m = site % SITES, cw = site / SITES;
    s_thr[i] = gtab_entry<GEO>(R.gJ, R.gS, cw / WR, cw % WR, m, p, beta_f);
  }
  const RoundKeys rk = make_round_keys(R.seed);
  fill_call_table<GEO, TPB>(s_tab, rk);
  const int r = (tid >> 5) * RW + (lane % RW);
  const int part = lane / RW;
  const int64_t slot = first + r;
  const bool live = slot < Rn;
  const int cur = R.cur, nxt = cur ^ 1;
  uint32_t* col = s_spin + r;
  if (live) {
    const int32_t src = R.src[slot];
    const uint4* p4 = reinterpret_cast<const uint4*>(R.spins[cur] + (size_t)src * W);
#pragma unroll 4
    for (int q = part; q < W / 4; q += P) {
      const uint4 v = p4[q];
      if (4 * q + 0 < WR) col[(4 * q + 0) * CS] = v.x;
      if (4 * q + 1 < WR) col[(4 * q + 1) * CS] = v.y;
      if (4 * q + 2 < WR) col[(4 * q + 2) * CS] = v.z;
      if (4 * q + 3 < WR) col[(4 * q + 3) * CS] = v.w;
    }
  }
  __syncthreads();
  GaussHalf gh;
  gh.slot = (uint32_t)slot;
  gh.seed = R.seed;
  gh.beta_f = beta_f;
  gh.bc = 0.0f;
  gh.lanes = __ballot_sync(0xFFFFFFFFu, live);
  gh.one = R.one;
  const uint32_t thr_base = (uint32_t)__cvta_generic_to_shared(s_thr);
  const int theta = R.theta_next;
  const uint32_t T0 = (uint32_t)R.sweeps;
  const int y0 = part * RPP;
  // half sweeps in chunks of NH tables, ordered as in k_sweep3d
  const int nhalf = 2 * theta;
#pragma unroll 1
  for (int h0 = 0; h0 < nhalf; h0 += SH::NH) {
    if (h0 > 0) __syncthreads();  // the previous chunk's tables are no longer read
    const int nh = min(SH::NH, nhalf - h0);
    build_half_tables<GEO, TPB, P>(s_tab, h0, nh, T0);
    if (live) {
#pragma unroll 1
      for (int j = 0; j < nh; ++j) {
        const uint32_t c = (uint32_t)j & 1u;  // h0 is even
        if (c == 0) {
          gh.T = T0 + (uint32_t)((h0 + j) >> 1);
          gh.key = sweep_key(gh.slot, gh.T, rk);
        }
        gh.c = c;
        gh.tag = TAG_SWEEP + c;
        gh.half = half_table<GEO, P>(s_tab, j) + part;
        if (P > 1 && j > 0) __syncwarp(gh.lanes);
        half_sweep_gtab3d<GEO, CS, RPP>(col, thr_base, gh, rk, y0);
      }
    }
  }
  __syncthreads();  // every row range swept before the energy reads its neighbour rows
  int E = 0;
  if (live) {
    int32_t anti = anti_rows_gauss3d<GEO, CS>(col, R.gJ, R.one, y0, y0 + RPP);
#pragma unroll
    for (int off = RW; off < 32; off <<= 1) anti += __shfl_xor_sync(gh.lanes, anti, off);
    E = R.gC0 - 2 * anti;
    uint4* d4 = reinterpret_cast<uint4*>(R.spins[nxt] + (size_t)slot * W);
#pragma unroll 4
    for (int q = part; q < W / 4; q += P) {
      uint4 v;
      v.x = (4 * q + 0 < WR) ? col[(4 * q + 0) * CS] : 0u;
      v.y = (4 * q + 1 < WR) ? col[(4 * q + 1) * CS] : 0u;
      v.z = (4 * q + 2 < WR) ? col[(4 * q + 2) * CS] : 0u;
      v.w = (4 * q + 3 < WR) ? col[(4 * q + 3) * CS] : 0u;
      d4[q] = v;
    }
  }
  measure_store_gauss(R, nxt, slot, live && part == 0, E);
}

template <int L, int TPB, int P>
cudaError_t launch_gtab3d_p(RunDev* runs, const Work* table, int nwork, cudaStream_t st) {
  if constexpr (!split_ok<Geo3<L>>(P) || TPB / P < 4 || (P > 1 && TPB < 64)) {
    return cudaErrorInvalidValue;
  } else {
    const size_t sm = sizeof(uint32_t) * GTabShape<L, TPB, P>::SMEM_WORDS;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute((const void*)k_sweep_gtab3d<L, TPB, P>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    if (nwork <= 0) return cudaSuccess;
    k_sweep_gtab3d<L, TPB, P><<<nwork * P, TPB, sm, st>>>(runs, table);
    return cudaGetLastError();
  }
}

// Blocks of 512 or 1024 threads: the sweep with threshold tables (the table
// build is shared by the block's replicas); the initial state as the other
// block sizes.
template <int L, int TPB>
cudaError_t launch_gtab3d_t(RunDev* runs, const Work* table, int nwork, cudaStream_t st, bool init, int split) {
  if (init) return launch_gauss3d_init<L, TPB>(runs, table, nwork, st);
  switch (split) {
    case 1: return launch_gtab3d_p<L, TPB, 1>(runs, table, nwork, st);
    case 2: return launch_gtab3d_p<L, TPB, 2>(runs, table, nwork, st);
    case 4: return launch_gtab3d_p<L, TPB, 4>(runs, table, nwork, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pa

// Edges with threshold tables: blocks of 32 .. 256 threads take the
// estimate-and-window kernel of pa_gauss3d.cuh, 512 and 1024 the tables.
#define PA_INSTANTIATE_GAUSS3D_TAB(LL)                                                                 \
  namespace pa {                                                                                       \
  cudaError_t launch_gauss3d_L##LL(int tpb, int split, RunDev* runs, const Work* table, int nwork,    \
                                   cudaStream_t st, bool init) {                                       \
    switch (tpb) {                                                                                     \
      case 32: return launch_gauss3d_t<LL, 32>(runs, table, nwork, st, init, split);                   \
      case 64: return launch_gauss3d_t<LL, 64>(runs, table, nwork, st, init, split);                   \
      case 128: return launch_gauss3d_t<LL, 128>(runs, table, nwork, st, init, split);                 \
      case 256: return launch_gauss3d_t<LL, 256>(runs, table, nwork, st, init, split);                 \
      case 512: return launch_gtab3d_t<LL, 512>(runs, table, nwork, st, init, split);                  \
      case 1024: return launch_gtab3d_t<LL, 1024>(runs, table, nwork, st, init, split);                \
      default: return cudaErrorInvalidValue;                                                           \
    }                                                                                                  \
  }                                                                                                    \
  bool gauss3d_split_ok_L##LL(int split) { return split <= 4 && split_ok<Geo3<LL>>(split); }          \
  }
