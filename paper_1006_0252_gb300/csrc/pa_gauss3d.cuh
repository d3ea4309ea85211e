// pa_gauss3d.cuh -- fused replica copy + checkerboard Metropolis sweeps +
// energy measurement for 3D periodic lattices with Gaussian couplings.
//
// Same replica layout, window and random keying as the +-1 kernel.  For a
// site i of colour c, with x_d = 1 where the spin of neighbour d differs from
// s_i (J s_i s_nb = -J there), the energy change of a flip is
//   dE_i = -2 sum_d J_d s_i s_nb = 4 sum_{d: x_d = 1} J_d - 2 S_i,
// S_i = sum_d J_d.  The couplings of the colour-c sites of a word are stored
// by rank m inside the word (gJ[c][d][w][m], gS[c][w][m]), so every shared
// memory index below is a compile-time offset from a per-word base.
#pragma once
#include "pa_gauss.cuh"
#include "pa_lattice3d.cuh"

namespace pa {

// Move the colour-c bits of a word to the even positions 2m (the inverse of
// to_colour_positions); other bits are discarded.
template <class GEO>
__device__ __forceinline__ uint32_t from_colour_positions(uint32_t v, uint32_t par0) {
  if constexpr ((GEO::G & 1) == 0) {
    return (v >> par0) & GEO::EVEN;
  } else {
    return (((v & GEO::LANES_EVEN) >> par0) | ((v & GEO::LANES_ODD) >> (par0 ^ 1u))) & GEO::EVEN;
  }
}

template <int K>
__device__ __forceinline__ int32_t lane4(const int4& v) {
  if constexpr (K == 0) return v.x;
  else if constexpr (K == 1) return v.y;
  else if constexpr (K == 2) return v.z;
  else return v.w;
}

// Energy change and windowed decision of the colour-c site of rank M (K = M
// mod 4 within the 128-bit groups jd, sv of couplings and sums).
template <int M, int K, int SITES, int A, int NU>
__device__ __forceinline__ void gauss_one(const uint32_t (&x)[6], const uint32_t (&u)[NU], const int4 (&jd)[6],
                                          const int4& sv, float bc, uint32_t one, uint32_t& flip, uint32_t& amb) {
  if constexpr (M < SITES) {
    int32_t acc = 0;
#pragma unroll
    for (int d = 0; d < 6; ++d) add_if_set<1u << (2 * M)>(acc, x[d], lane4<K>(jd[d]), one);
    gauss_site(4 * acc - 2 * lane4<K>(sv), bc, u[A + M], 1u << (2 * M), one, &flip, &amb);
  }
}

// Ranks 4 M4 .. 4 M4 + 3 of a word, then the next group (compile-time loop).
template <int SITES, int A, int DSTRIDE4, int M4, int NM4, int NU>
__device__ __forceinline__ void gauss_word_sites(const uint32_t (&x)[6], const uint32_t (&u)[NU],
                                                 const int4* __restrict__ Jw4, const int4* __restrict__ Sw4, float bc,
                                                 uint32_t one, uint32_t& flip, uint32_t& amb) {
  if constexpr (M4 < NM4) {
    int4 jd[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) jd[d] = Jw4[d * DSTRIDE4 + M4];
    const int4 sv = Sw4[M4];
    gauss_one<4 * M4 + 0, 0, SITES, A>(x, u, jd, sv, bc, one, flip, amb);
    gauss_one<4 * M4 + 1, 1, SITES, A>(x, u, jd, sv, bc, one, flip, amb);
    gauss_one<4 * M4 + 2, 2, SITES, A>(x, u, jd, sv, bc, one, flip, amb);
    gauss_one<4 * M4 + 3, 3, SITES, A>(x, u, jd, sv, bc, one, flip, amb);
    gauss_word_sites<SITES, A, DSTRIDE4, M4 + 1, NM4>(x, u, Jw4, Sw4, bc, one, flip, amb);
  }
}

// Exact decisions (gauss_accept) for the sites of one word whose uniform fell
// inside the estimate's window: bit 2m of amb for rank m.  Rare, so the
// uniform is regenerated and the energy change recomputed here, out of line.
static __device__ __noinline__ uint32_t gauss_resolve(uint32_t amb, uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3,
                                               uint32_t x4, uint32_t x5, const int32_t* __restrict__ Jw,
                                               const int32_t* __restrict__ Sw, int dstride, uint32_t r0,
                                               uint32_t slot, uint32_t T, uint32_t tag, uint64_t seed,
                                               float beta_f) {
  const uint32_t x[6] = {x0, x1, x2, x3, x4, x5};
  uint32_t res = 0u;
  while (amb) {
    const int bit = __ffs(amb) - 1;
    const int m = bit >> 1;
    const uint32_t rank = r0 + (uint32_t)m;  // colour-c rank of the site
    const u32x4 v = philox_seeded(seed, rank >> 2, slot, T, tag);
    const uint32_t u = pick(v, (int)(rank & 3u));
    int32_t acc = 0;
    for (int d = 0; d < 6; ++d)
      if ((x[d] >> bit) & 1u) acc += Jw[d * dstride + m];
    const int32_t dE = 4 * acc - 2 * Sw[m];
    if (gauss_accept(dE, beta_f, u)) res |= 1u << bit;
    amb &= amb - 1u;
  }
  return res;
}

// Word g of row y (the Gaussian counterpart of word3d): anti-alignment
// masks, the word's uniforms (alignment A, shared calls in `carry`), per-site
// energy changes and decisions, and the out-of-line exact path.
// Everything a word's update needs beyond the lattice: the half-sweep table
// and the slot's key (uniforms), the counter words and seed (the exact path
// regenerates a uniform directly), beta, and the live lanes of the warp.
struct GaussHalf {
  const uint4* half;
  SweepKey key;
  uint32_t slot, T, c, tag;
  uint64_t seed;
  float beta_f, bc;
  unsigned lanes;
  uint32_t one;
};

template <class GEO, int A>
__device__ __forceinline__ void gword3d(int g, int y, const int32_t* __restrict__ s_J, const int32_t* __restrict__ s_S,
                                        uint32_t (&rowm)[GEO::G], uint32_t (&row)[GEO::G],
                                        const uint32_t (&rowp)[GEO::G], const GaussHalf& gh, const RoundKeys& rk,
                                        uint32_t (&carry)[4]) {
  constexpr int G = GEO::G, L = GEO::L, K = GEO::K, WR = GEO::WR;
  constexpr int SITES = K * L / 2, SP = (SITES + 3) & ~3;
  const int w = y * G + g;
  const uint32_t s = row[g];
  const uint32_t c = gh.c, one = gh.one;
  const uint32_t par0 = (c + (uint32_t)y + (uint32_t)g) & 1u;
  const uint32_t zp = (g + 1 < G) ? row[(g + 1) % G] : lanes_down<GEO>(row[0]);
  const uint32_t zm = (g > 0) ? row[(g + G - 1) % G] : lanes_up<GEO>(row[G - 1]);
  uint32_t x[6];
  x[0] = from_colour_positions<GEO>(s ^ rot_xp<GEO>(s), par0);
  x[1] = from_colour_positions<GEO>(s ^ rot_xm<GEO>(s), par0);
  x[2] = from_colour_positions<GEO>(s ^ rowp[g], par0);
  x[3] = from_colour_positions<GEO>(s ^ rowm[g], par0);
  x[4] = from_colour_positions<GEO>(s ^ zp, par0);
  x[5] = from_colour_positions<GEO>(s ^ zm, par0);
  const uint32_t r0 = (uint32_t)(w * SITES);  // colour-c rank of the word's first site
  uint32_t u[4 * word_calls<SITES, A>()];
  word_uniforms<SITES, A>(r0 >> 2, gh.half, gh.key, rk, carry, u);
  const int32_t* Jw = s_J + (c * 6 * WR + w) * SP;  // direction d at + d * WR * SP
  const int32_t* Sw = s_S + (c * WR + w) * SP;
  const int4* Jw4 = reinterpret_cast<const int4*>(Jw);
  const int4* Sw4 = reinterpret_cast<const int4*>(Sw);
  uint32_t flip = 0u, amb = 0u;
  gauss_word_sites<SITES, A, WR * SP / 4, 0, SP / 4>(x, u, Jw4, Sw4, gh.bc, one, flip, amb);
  if (__any_sync(gh.lanes, amb != 0u))
    flip |= gauss_resolve(amb, x[0], x[1], x[2], x[3], x[4], x[5], Jw, Sw, WR * SP, r0, gh.slot, gh.T, gh.tag,
                          gh.seed, gh.beta_f);
  row[g] = s ^ to_colour_positions<GEO>(flip, par0);
}

template <class GEO, int CS, int YP>
__device__ __forceinline__ void grow3d(uint32_t* __restrict__ col, const int32_t* __restrict__ s_J,
                                       const int32_t* __restrict__ s_S, int y, uint32_t (&rowm)[GEO::G],
                                       uint32_t (&row)[GEO::G], uint32_t (&rowp)[GEO::G], const GaussHalf& gh,
                                       const RoundKeys& rk, uint32_t (&carry)[4]) {
  constexpr int G = GEO::G, L = GEO::L, K = GEO::K;
  constexpr int SITES = K * L / 2;
  const int yn = (y + 1 == L) ? 0 : y + 1;
#pragma unroll
  for (int g = 0; g < G; ++g) rowp[g] = col[(yn * G + g) * CS];
  if constexpr (SITES % 4 == 0) {
#pragma unroll
    for (int g = 0; g < G; ++g) gword3d<GEO, 0>(g, y, s_J, s_S, rowm, row, rowp, gh, rk, carry);
  } else {
    static_for<0, G>([&](auto gc) {
      constexpr int g = decltype(gc)::value;
      constexpr int A = (SITES * (YP * G + g)) % 4;
      gword3d<GEO, A>(g, y, s_J, s_S, rowm, row, rowp, gh, rk, carry);
    });
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    col[(y * G + g) * CS] = row[g];
    rowm[g] = row[g];
    row[g] = rowp[g];
  }
}

// One Metropolis half sweep over the colour-c sites of the RPP rows y0 ..
// y0 + RPP - 1 of one replica.  Per word: the six anti-alignment masks, the
// word's uniforms, then per site the energy change from the shared-memory
// couplings (four ranks per 128-bit load) and the branch-free windowed
// decision; sites inside the window are settled by gauss_resolve under a
// warp-uniform branch.  Rows go in pairs when the colour-c sites per word are
// not a multiple of 4 (see row3d in pa_sweep3d.cuh).
template <class GEO, int CS, int RPP>
__device__ __forceinline__ void half_sweep_gauss3d(uint32_t* __restrict__ col, const int32_t* __restrict__ s_J,
                                                   const int32_t* __restrict__ s_S, const GaussHalf& gh,
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
    for (int i = 0; i < RPP; ++i) grow3d<GEO, CS, 0>(col, s_J, s_S, y0 + i, rowm, row, rowp, gh, rk, carry);
  } else {
    static_assert(RPP % 2 == 0, "rows come in pairs");
#pragma unroll 1
    for (int i = 0; i < RPP; i += 2) {
      grow3d<GEO, CS, 0>(col, s_J, s_S, y0 + i, rowm, row, rowp, gh, rk, carry);
      grow3d<GEO, CS, 1>(col, s_J, s_S, y0 + i + 1, rowm, row, rowp, gh, rk, carry);
    }
  }
}

// Energy in fixed-point units: E = C0 - 2 sum over "+" bonds with x = 1 of J,
// C0 = sum of all couplings; both colours of every word.
template <class GEO, int TPB>
__device__ __forceinline__ int32_t anti_rows_gauss3d(const uint32_t* __restrict__ col, const int32_t* __restrict__ s_J,
                                                     uint32_t one, int y0, int y1) {
  constexpr int G = GEO::G, L = GEO::L, K = GEO::K, WR = GEO::WR;
  constexpr int SITES = K * L / 2, SP = (SITES + 3) & ~3;
  int32_t anti = 0;
  for (int y = y0; y < y1; ++y) {
    const int yn = (y + 1 == L) ? 0 : y + 1;
    uint32_t row[G], rowp[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      row[g] = col[(y * G + g) * TPB];
      rowp[g] = col[(yn * G + g) * TPB];
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int w = y * G + g;
      const uint32_t s = row[g];
      const uint32_t zp = (g + 1 < G) ? row[(g + 1) % G] : lanes_down<GEO>(row[0]);
      const uint32_t ax = s ^ rot_xp<GEO>(s), ay = s ^ rowp[g], az = s ^ zp;
#pragma unroll
      for (uint32_t c = 0; c < 2; ++c) {
        const uint32_t par0 = (c + (uint32_t)y + (uint32_t)g) & 1u;
        const uint32_t x0 = from_colour_positions<GEO>(ax, par0);
        const uint32_t x2 = from_colour_positions<GEO>(ay, par0);
        const uint32_t x4 = from_colour_positions<GEO>(az, par0);
        const int32_t* Jw = s_J + (c * 6 * WR + w) * SP;
#pragma unroll
        for (int m = 0; m < SITES; ++m) {
          add_if_set(anti, x0, 1u << (2 * m), Jw[0 * WR * SP + m], one);
          add_if_set(anti, x2, 1u << (2 * m), Jw[2 * WR * SP + m], one);
          add_if_set(anti, x4, 1u << (2 * m), Jw[4 * WR * SP + m], one);
        }
      }
    }
  }
  return anti;
}

template <class GEO, int TPB>
__device__ __forceinline__ int energy_gauss3d(const uint32_t* __restrict__ col, const int32_t* __restrict__ s_J,
                                              int32_t C0, uint32_t one) {
  return C0 - 2 * anti_rows_gauss3d<GEO, TPB>(col, s_J, one, 0, GEO::L);
}

__device__ __forceinline__ void measure_store_gauss(RunDev& R, int nxt, int64_t slot, bool live, int E) {
  long long e = 0ll;
  unsigned long long lo = 0ull, hi = 0ull;
  if (live) {
    R.E[nxt][slot] = E;
    atomicMin(&R.emin_next, (long long)E);
    e = E;
    const unsigned long long q = (unsigned long long)((long long)E * (long long)E);  // < 2^62
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

// Per-site table words: [2][6][WR][SP] couplings + [2][WR][SP] sums, SP = the
// colour-c sites per word rounded up to a multiple of 4 (16-byte rows).
template <int L>
__host__ __device__ constexpr size_t gauss_tables_words() {
  return 14 * (size_t)Geo3<L>::WR * (((Geo3<L>::K * L / 2) + 3) & ~3);
}

// Replicas per block TPB / P; see SweepShape in pa_sweep3d.cuh.
template <int L, int TPB, int P>
struct GaussShape {
  using GEO = Geo3<L>;
  static constexpr int NR = TPB / P;
  static constexpr int RPP = L / P;
  static constexpr int CS = split_stride(NR, RPP * GEO::G, P, TPB);
  static constexpr int NH = half_tables<GEO, TPB, P>(4 * (gauss_tables_words<L>() + GEO::WR * CS));
  static constexpr size_t SMEM_WORDS =
      gauss_tables_words<L>() + (size_t)sweep_table_words<GEO, P>(NH) + (size_t)GEO::WR * CS;
};

// Sec. 2 with the Gaussian couplings of Sec. 4: gather of the resampled
// population, theta checkerboard sweeps at beta', and the energy of every
// replica; P threads per replica on ranges of whole rows (block b takes work
// item b / P of the class table and its (b mod P)-th share).
template <int L, int TPB, int P>
__global__ void __launch_bounds__(TPB) k_sweep_gauss3d(RunDev* __restrict__ runs, const Work* __restrict__ table) {
  using GEO = Geo3<L>;
  using SH = GaussShape<L, TPB, P>;
  constexpr int WR = GEO::WR, W = GEO::W, SP = ((GEO::K * L / 2) + 3) & ~3;
  constexpr int NJ = 2 * 6 * WR * SP, NS = 2 * WR * SP;
  constexpr int RW = 32 / P, RPP = SH::RPP, CS = SH::CS;
  extern __shared__ __align__(16) uint32_t smem[];
  uint4* s_tab = reinterpret_cast<uint4*>(smem);  // sweep_table_words
  int32_t* s_J = reinterpret_cast<int32_t*>(smem + sweep_table_words<GEO, P>(SH::NH));
  int32_t* s_S = s_J + NJ;
  uint32_t* s_spin = reinterpret_cast<uint32_t*>(s_S + NS);
  const Work wk = table[blockIdx.x / P];
  RunDev& R = runs[wk.run];
  if (R.skip) return;
  const int64_t Rn = R.R_next;
  const int64_t first = (int64_t)wk.first + (int64_t)(blockIdx.x % P) * SH::NR;
  if (first >= Rn) return;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < NJ; i += TPB) s_J[i] = R.gJ[i];
  for (int i = tid; i < NS; i += TPB) s_S[i] = R.gS[i];
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
  gh.beta_f = __double2float_rn(R.beta_next);
  gh.bc = __fmul_rn(gh.beta_f, GAUSS_LOG2E_SCALED);
  gh.lanes = __ballot_sync(0xFFFFFFFFu, live);
  gh.one = R.one;
  const int theta = R.theta_next;
  const uint32_t T0 = (uint32_t)R.sweeps;
  const int y0 = part * RPP;
  // half sweeps in chunks of NH tables, ordered as in k_sweep3d: block
  // barriers around each chunk's tables, a warp barrier between the half
  // sweeps of a replica's P threads within a chunk
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
        half_sweep_gauss3d<GEO, CS, RPP>(col, s_J, s_S, gh, rk, y0);
      }
    }
  }
  __syncthreads();  // every row range swept before the energy reads its neighbour rows
  int E = 0;
  if (live) {
    int32_t anti = anti_rows_gauss3d<GEO, CS>(col, s_J, R.one, y0, y0 + RPP);
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

// Sec. 2: R0 independent uniformly random microstates at beta = 0 (keying as
// k_init3d) and their fixed-point energies.
template <int L, int TPB>
__global__ void __launch_bounds__(TPB) k_init_gauss3d(RunDev* __restrict__ runs, const Work* __restrict__ table) {
  using GEO = Geo3<L>;
  constexpr int WR = GEO::WR, W = GEO::W, SP = ((GEO::K * L / 2) + 3) & ~3;
  constexpr int NJ = 2 * 6 * WR * SP;
  extern __shared__ __align__(16) uint32_t smem[];
  int32_t* s_J = reinterpret_cast<int32_t*>(smem);
  uint32_t* s_spin = smem + gauss_tables_words<L>();
  const Work wk = table[blockIdx.x];
  RunDev& R = runs[wk.run];
  const int64_t R0 = R.R;
  if ((int64_t)wk.first >= R0) return;
  const int tid = threadIdx.x;
  for (int i = tid; i < NJ; i += TPB) s_J[i] = R.gJ[i];
  const int64_t slot = (int64_t)wk.first + tid;
  const bool live = slot < R0;
  uint32_t* col = s_spin + tid;
  if (live) {
    for (int w4 = 0; w4 < W / 4; ++w4) {
      const u32x4 u = philox_seeded(R.seed, (uint32_t)w4, (uint32_t)slot, 0u, TAG_INIT);
      if (4 * w4 + 0 < WR) col[(4 * w4 + 0) * TPB] = u.a & GEO::VALID;
      if (4 * w4 + 1 < WR) col[(4 * w4 + 1) * TPB] = u.b & GEO::VALID;
      if (4 * w4 + 2 < WR) col[(4 * w4 + 2) * TPB] = u.c & GEO::VALID;
      if (4 * w4 + 3 < WR) col[(4 * w4 + 3) * TPB] = u.d & GEO::VALID;
    }
  }
  __syncthreads();
  int E = 0;
  if (live) {
    E = energy_gauss3d<GEO, TPB>(col, s_J, R.gC0, R.one);
    store_column<GEO, TPB>(R.spins[0] + (size_t)slot * W, col);
  }
  measure_store_gauss(R, 0, slot, live, E);
}

template <int L, int TPB, int P>
cudaError_t launch_gauss3d_p(RunDev* runs, const Work* table, int nwork, cudaStream_t st) {
  if constexpr (!split_ok<Geo3<L>>(P) || TPB / P < 4 || (P > 1 && TPB < 64)) {
    return cudaErrorInvalidValue;
  } else {
    const size_t sm = sizeof(uint32_t) * GaussShape<L, TPB, P>::SMEM_WORDS;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute((const void*)k_sweep_gauss3d<L, TPB, P>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    if (nwork <= 0) return cudaSuccess;
    k_sweep_gauss3d<L, TPB, P><<<nwork * P, TPB, sm, st>>>(runs, table);
    return cudaGetLastError();
  }
}

template <int L, int TPB>
cudaError_t launch_gauss3d_init(RunDev* runs, const Work* table, int nwork, cudaStream_t st) {
  using GEO = Geo3<L>;
  const size_t sm = 4 * (gauss_tables_words<L>() + (size_t)GEO::WR * TPB);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_init_gauss3d<L, TPB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (nwork <= 0) return cudaSuccess;
  k_init_gauss3d<L, TPB><<<nwork, TPB, sm, st>>>(runs, table);
  return cudaGetLastError();
}

template <int L, int TPB>
cudaError_t launch_gauss3d_t(RunDev* runs, const Work* table, int nwork, cudaStream_t st, bool init, int split) {
  if (init) return launch_gauss3d_init<L, TPB>(runs, table, nwork, st);
  switch (split) {
    case 1: return launch_gauss3d_p<L, TPB, 1>(runs, table, nwork, st);
    case 2: return launch_gauss3d_p<L, TPB, 2>(runs, table, nwork, st);
    case 4: return launch_gauss3d_p<L, TPB, 4>(runs, table, nwork, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pa

#define PA_INSTANTIATE_GAUSS3D(LL)                                                                     \
  namespace pa {                                                                                       \
  cudaError_t launch_gauss3d_L##LL(int tpb, int split, RunDev* runs, const Work* table, int nwork,    \
                                   cudaStream_t st, bool init) {                                       \
    switch (tpb) {                                                                                     \
      case 32: return launch_gauss3d_t<LL, 32>(runs, table, nwork, st, init, split);                   \
      case 64: return launch_gauss3d_t<LL, 64>(runs, table, nwork, st, init, split);                   \
      case 128: return launch_gauss3d_t<LL, 128>(runs, table, nwork, st, init, split);                 \
      case 256: return launch_gauss3d_t<LL, 256>(runs, table, nwork, st, init, split);                 \
      default: return cudaErrorInvalidValue;                                                           \
    }                                                                                                  \
  }                                                                                                    \
  bool gauss3d_split_ok_L##LL(int split) { return split <= 4 && split_ok<Geo3<LL>>(split); }          \
  }
