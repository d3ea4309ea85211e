// pa_sweep3d.cuh -- fused replica copy + checkerboard Metropolis sweeps +
// energy measurement for 3D periodic cubic +-1 spin glasses (Sec. 2: "all
// replicas are now subject to an equilibrating MCMC process at the new
// temperature"; Algorithm: "Equilibrate replica j for theta sweeps", then
// "Compute observables").
//
// P threads own one replica (P = 1, 2, 4 or 8, chosen per lattice class).
// The replica's packed words live in a column of shared memory (word w of
// replica r at s_spin[w * CS + r], so a warp touches consecutive banks); each
// thread sweeps its L / P y-rows with a three-row sliding window in registers
// and updates the G words of a row with 32-bit bitwise logic: for every
// direction d the bond bit b_d = s ^ s_nb ^ j_d is 1 where the bond is
// satisfied (J s s' = -1), a carry-save adder counts the n satisfied bonds per
// site (dE = 4n - 12), and a site flips iff n <= 3 or its uniform
// u < threshold[dE/2] (only energy rises draw on the uniform).
#pragma once
#include "pa_lattice3d.cuh"

namespace pa {

// Bond masks of one run: [6][W] words; direction order x+, x-, y+, y-, z+, z-;
// bit (w, p) set iff the coupling of that bond of site (w, p) is -1.
enum { DXP = 0, DXM = 1, DYP = 2, DYM = 3, DZP = 4, DZM = 5 };

// Satisfied-bond counts of the "+" bonds of one word (energy measurement).
template <class GEO>
__device__ __forceinline__ int plus_bonds_satisfied(uint32_t s, uint32_t yp, uint32_t zp, uint32_t jxp, uint32_t jyp,
                                                    uint32_t jzp) {
  const uint32_t bx = s ^ rot_xp<GEO>(s) ^ jxp;
  const uint32_t by = s ^ yp ^ jyp;
  const uint32_t bz = s ^ zp ^ jzp;
  return __popc(bx & GEO::VALID) + __popc(by & GEO::VALID) + __popc(bz & GEO::VALID);
}

// Satisfied "+" bonds of rows y0 .. y1-1 of the replica in a shared-memory
// column (word w at col[w * CS]).
template <class GEO, int CS>
__device__ __forceinline__ int satisfied_rows(const uint32_t* __restrict__ col, const uint32_t* __restrict__ s_bond,
                                              int y0, int y1) {
  constexpr int G = GEO::G, L = GEO::L, W = GEO::W;
  int sat = 0;
  for (int y = y0; y < y1; ++y) {
    const int yn = (y + 1 == L) ? 0 : y + 1;
    uint32_t row[G], rowp[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      row[g] = col[(y * G + g) * CS];
      rowp[g] = col[(yn * G + g) * CS];
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int w = y * G + g;
      const uint32_t zp = (g + 1 < G) ? row[(g + 1) % G] : lanes_down<GEO>(row[0]);
      sat += plus_bonds_satisfied<GEO>(row[g], rowp[g], zp, s_bond[DXP * W + w], s_bond[DYP * W + w],
                                       s_bond[DZP * W + w]);
    }
  }
  return sat;
}

// Record energy, histogram and exact sums of one replica (lanes with
// live == false contribute nothing but take part in the warp reduction).
__device__ __forceinline__ void measure_store(RunDev& R, int nxt, int64_t slot, bool live, int E) {
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

// ---------------------------------------------------------------------------
// Threshold compares.  Bit m of ge is [u_m >= thr]: the subtraction u_m - thr
// sets the carry exactly when it does not borrow, and ge = 2 ge + carry
// shifts it in (two integer instructions per site); the complement is then
// spread from bit m to bit 2m, the position mask layout of the word.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t spread_even(uint32_t x) {  // bit m -> bit 2m, m < 16
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

template <int SITES, int OFF>
__device__ __forceinline__ uint32_t lt_mask(const uint32_t* u, uint32_t thr) {
  static_assert(SITES <= 16, "at most 16 colour-c sites per word");
  uint32_t ge = 0u;
#pragma unroll
  for (int m = SITES - 1; m >= 0; --m)
    asm("{\n\t.reg .u32 t;\n\tsub.cc.u32 t, %1, %2;\n\taddc.u32 %0, %3, %3;\n\t}"
        : "=r"(ge)
        : "r"(u[OFF + m]), "r"(thr), "r"(ge));
  constexpr uint32_t VM = (1u << SITES) - 1u;
  return spread_even(~ge & VM);
}

// The compares with thr(4) and thr(8) in one chain (at high temperature both
// are needed for almost every word): per site two subtractions shift their
// carries in, so bit 2m+1 = [u_m >= thr4] and bit 2m = [u_m >= thr8], and no
// spreading is needed.
template <int SITES, int OFF>
__device__ __forceinline__ void lt_mask2(const uint32_t* u, uint32_t thr4, uint32_t thr8, uint32_t& e4,
                                         uint32_t& e8) {
  static_assert(SITES <= 16, "at most 16 colour-c sites per word");
  uint32_t ge = 0u;
#pragma unroll
  for (int m = SITES - 1; m >= 0; --m)
    asm("{\n\t.reg .u32 t;\n\tsub.cc.u32 t, %1, %2;\n\taddc.u32 %0, %4, %4;\n\t"
        "sub.cc.u32 t, %1, %3;\n\taddc.u32 %0, %0, %0;\n\t}"
        : "=r"(ge)
        : "r"(u[OFF + m]), "r"(thr4), "r"(thr8), "r"(ge));
  constexpr uint32_t EV = (2 * SITES >= 32) ? 0x55555555u : (0x55555555u & ((1u << (2 * SITES)) - 1u));
  e4 = (~ge >> 1) & EV;
  e8 = ~ge & EV;
}

// Everything a word's update needs beyond the lattice: the half-sweep table,
// the slot's key, the colour and the thresholds of dE = 4, 8, 12.
struct HalfSweep {
  const uint4* half;
  SweepKey key;
  uint32_t c;
  uint32_t T4, T8, T12;
  bool low_t;      // T4 < 2^22: most words draw no uniform below T4
  bool high_t;     // T4 >= 2^24: almost every word needs the compares with T4 and T8
  unsigned lanes;  // live lanes of the warp
};

// Compares of the word's uniforms with the thresholds of dE = 4, 8, 12
// (masks at even positions 2m: bit set iff u_m < thr).  thr4 >= thr8 >= thr12,
// so where u >= thr4 the other two compares fail as well: they are skipped for
// the word when no lane of the warp has a uniform below thr4.  At low
// temperature the uniforms are first reduced to their minimum, and the word
// skips all compares when no lane's minimum is below thr4; at high
// temperature the compares with thr4 and thr8 run as one chain (lt_mask2).
// Minimum of u[OFF .. OFF+N-1], folded three at a time.
template <int N, int OFF>
__device__ __forceinline__ uint32_t min_of(const uint32_t* u) {
  if constexpr (N == 1) {
    return u[OFF];
  } else if constexpr (N == 2) {
    return min(u[OFF], u[OFF + 1]);
  } else {
    constexpr int H = N / 3, R = N - 2 * H;
    return min(min(min_of<H, OFF>(u), min_of<H, OFF + H>(u)), min_of<R, OFF + 2 * H>(u));
  }
}

// Returns false when no lane of the warp can have a uniform below thr4 in this
// word (then the masks are zero and the caller takes the plain update).
template <int SITES, int A>
__device__ __forceinline__ bool word_compares(uint32_t q0, const HalfSweep& hs, const RoundKeys& rk,
                                              uint32_t (&carry)[4], uint32_t& e4, uint32_t& e8, uint32_t& e12) {
  uint32_t u[4 * word_calls<SITES, A>()];
  word_uniforms<SITES, A>(q0, hs.half, hs.key, rk, carry, u);
  e4 = 0u;
  e8 = 0u;
  e12 = 0u;
  if (hs.low_t) {
    if (!__any_sync(hs.lanes, min_of<SITES, A>(u) < hs.T4)) return false;
  }
  if (hs.high_t) {
    lt_mask2<SITES, A>(u, hs.T4, hs.T8, e4, e8);
  } else {
    e4 = lt_mask<SITES, A>(u, hs.T4);
    if (!__any_sync(hs.lanes, e4 != 0u)) return false;
    e8 = lt_mask<SITES, A>(u, hs.T8);
  }
  if (__any_sync(hs.lanes, e8 != 0u)) e12 = lt_mask<SITES, A>(u, hs.T12);
  return true;
}

// Word g of row y: bond bits, satisfied-bond count, compares, flips.  A is
// the alignment of the word's first uniform (see word_uniforms).
template <class GEO, int A>
__device__ __forceinline__ void word3d(int g, int y, const uint32_t* __restrict__ s_bond, uint32_t (&rowm)[GEO::G],
                                       uint32_t (&row)[GEO::G], const uint32_t (&rowp)[GEO::G], const HalfSweep& hs,
                                       const RoundKeys& rk, uint32_t (&carry)[4]) {
  constexpr int G = GEO::G, L = GEO::L, W = GEO::W, K = GEO::K;
  constexpr int SITES = K * L / 2;  // colour-c sites per word
  const int w = y * G + g;
  const uint32_t s = row[g];
  const uint32_t zp = (g + 1 < G) ? row[(g + 1) % G] : lanes_down<GEO>(row[0]);
  const uint32_t zm = (g > 0) ? row[(g + G - 1) % G] : lanes_up<GEO>(row[G - 1]);
  const uint32_t b0 = s ^ rot_xp<GEO>(s) ^ s_bond[DXP * W + w];
  const uint32_t b1 = s ^ rot_xm<GEO>(s) ^ s_bond[DXM * W + w];
  const uint32_t b2 = s ^ rowp[g] ^ s_bond[DYP * W + w];
  const uint32_t b3 = s ^ rowm[g] ^ s_bond[DYM * W + w];
  const uint32_t b4 = s ^ zp ^ s_bond[DZP * W + w];
  const uint32_t b5 = s ^ zm ^ s_bond[DZM * W + w];
  // carry-save count of the six bond bits: n = 4 n2 + 2 n1 + n0
  const uint32_t sa = b0 ^ b1 ^ b2, ca = (b0 & b1) | (b2 & (b0 ^ b1));
  const uint32_t sb = b3 ^ b4 ^ b5, cb = (b3 & b4) | (b5 & (b3 ^ b4));
  const uint32_t n0 = sa ^ sb, c0 = sa & sb;
  const uint32_t n1 = ca ^ cb ^ c0, n2 = (ca & cb) | (c0 & (ca ^ cb));
  uint32_t e4, e8, e12;
  const bool drawn = word_compares<SITES, A>((uint32_t)(w * SITES) >> 2, hs, rk, carry, e4, e8, e12);
  const uint32_t par0 = (hs.c + (uint32_t)y + (uint32_t)g) & 1u;
  const uint32_t cm = to_colour_positions<GEO>(GEO::EVEN, par0);
  if (!drawn) {  // warp-uniform: no rise accepted in this word, only n <= 3 sites flip
    row[g] = s ^ (cm & ~n2);
    return;
  }
  const uint32_t a4 = to_colour_positions<GEO>(e4, par0);
  const uint32_t a8 = to_colour_positions<GEO>(e8, par0);
  const uint32_t a12 = to_colour_positions<GEO>(e12, par0);
  // n = 4, 5, 6 take the compare with thr(4), thr(8), thr(12)
  const uint32_t sel = (n1 & a12) | (~n1 & ((n0 & a8) | (~n0 & a4)));
  row[g] = s ^ (cm & (~n2 | sel));
}

// Row y of a half sweep (three-row window rowm / row / rowp).  YP is the
// row's position in its pair of rows (y mod 2 when SITES is not a multiple of
// 4): a pair of rows holds L^2/2 sites of each colour, a multiple of 4, so
// the alignment of every word's first uniform is known at compile time.
template <class GEO, int CS, int YP>
__device__ __forceinline__ void row3d(uint32_t* __restrict__ col, const uint32_t* __restrict__ s_bond, int y,
                                      uint32_t (&rowm)[GEO::G], uint32_t (&row)[GEO::G], uint32_t (&rowp)[GEO::G],
                                      const HalfSweep& hs, const RoundKeys& rk, uint32_t (&carry)[4]) {
  constexpr int G = GEO::G, L = GEO::L, K = GEO::K;
  constexpr int SITES = K * L / 2;
  const int yn = (y + 1 == L) ? 0 : y + 1;
#pragma unroll
  for (int g = 0; g < G; ++g) rowp[g] = col[(yn * G + g) * CS];
  if constexpr (SITES % 4 == 0) {
#pragma unroll
    for (int g = 0; g < G; ++g) word3d<GEO, 0>(g, y, s_bond, rowm, row, rowp, hs, rk, carry);
  } else {
    static_for<0, G>([&](auto gc) {
      constexpr int g = decltype(gc)::value;
      constexpr int A = (SITES * (YP * G + g)) % 4;
      word3d<GEO, A>(g, y, s_bond, rowm, row, rowp, hs, rk, carry);
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
// y0 + RPP - 1 of one replica (whole pairs of rows when SITES is not a
// multiple of 4).  Ranges of at most two rows are unrolled.
template <class GEO, int CS, int RPP>
__device__ __forceinline__ void half_sweep3d(uint32_t* __restrict__ col, const uint32_t* __restrict__ s_bond,
                                             const HalfSweep& hs, const RoundKeys& rk, int y0) {
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
    if constexpr (RPP <= 2) {
#pragma unroll
      for (int i = 0; i < RPP; ++i) row3d<GEO, CS, 0>(col, s_bond, y0 + i, rowm, row, rowp, hs, rk, carry);
    } else {
#pragma unroll 1
      for (int i = 0; i < RPP; ++i) row3d<GEO, CS, 0>(col, s_bond, y0 + i, rowm, row, rowp, hs, rk, carry);
    }
  } else {
    static_assert(RPP % 2 == 0, "rows come in pairs");
#pragma unroll 1
    for (int i = 0; i < RPP; i += 2) {
      row3d<GEO, CS, 0>(col, s_bond, y0 + i, rowm, row, rowp, hs, rk, carry);
      row3d<GEO, CS, 1>(col, s_bond, y0 + i + 1, rowm, row, rowp, hs, rk, carry);
    }
  }
}

// Replicas per block: TPB / P; block b takes work item b / P of the class
// table (TPB consecutive slots of one run) and its (b mod P)-th share.
template <int L, int TPB, int P>
struct SweepShape {
  using GEO = Geo3<L>;
  static constexpr int NR = TPB / P;                                    // replicas per block
  static constexpr int RPP = L / P;                                     // rows per thread
  static constexpr int CS = split_stride(NR, RPP * GEO::G, P, TPB);     // column stride
  // half-sweep tables held at once: with one thread per replica as many as
  // fit; with several, two, double-buffered (one block barrier per half
  // sweep measured 1 % faster at L = 8 with four threads per replica than
  // chunks of tables with warp barriers between their half sweeps)
  static constexpr int NH = P > 1 ? 2 : half_tables<GEO, TPB, P>(4 * (6 * GEO::W + GEO::WR * CS));
  static constexpr int SMEM_WORDS = sweep_table_words<GEO, P>(NH) + 6 * GEO::W + GEO::WR * CS;
};

// Sec. 2: the gather of the resampled population (slot s <- old slot src(s)),
// theta checkerboard sweeps at beta', and the energy of every replica.
template <int L, int TPB, int P>
__global__ void __launch_bounds__(TPB) k_sweep3d(RunDev* __restrict__ runs, const Work* __restrict__ table) {
  using GEO = Geo3<L>;
  using SH = SweepShape<L, TPB, P>;
  constexpr int WR = GEO::WR, W = GEO::W, RW = 32 / P, RPP = SH::RPP, CS = SH::CS;
  extern __shared__ __align__(16) uint32_t smem[];
  uint4* s_tab = reinterpret_cast<uint4*>(smem);             // sweep_table_words
  uint32_t* s_bond = smem + sweep_table_words<GEO, P>(SH::NH);  // [6][W]
  uint32_t* s_spin = s_bond + 6 * W;                  // [WR][CS]
  const Work wk = table[blockIdx.x / P];
  RunDev& R = runs[wk.run];
  if (R.skip) return;
  const int64_t Rn = R.R_next;
  const int64_t first = (int64_t)wk.first + (int64_t)(blockIdx.x % P) * SH::NR;
  if (first >= Rn) return;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < 6 * W; i += TPB) s_bond[i] = R.bonds[i];
  const RoundKeys rk = make_round_keys(R.seed);
  fill_call_table<GEO, TPB>(s_tab, rk);
  const int r = (tid >> 5) * RW + (lane % RW);  // replica of this thread in the block
  const int part = lane / RW;                   // its row range
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
  HalfSweep hs;
  hs.T4 = R.thr[2];
  hs.T8 = R.thr[4];
  hs.T12 = R.thr[6];
  hs.low_t = hs.T4 < (1u << 22);
  hs.high_t = hs.T4 >= (1u << 24);
  hs.lanes = __ballot_sync(0xFFFFFFFFu, live);
  const int theta = R.theta_next;
  const uint32_t T0 = (uint32_t)R.sweeps;
  const int y0 = part * RPP;
  if constexpr (P > 1) {
    // several threads per replica: one table per half sweep, double-buffered,
    // behind a block barrier that also orders the row ranges' half sweeps (a
    // colour-c half sweep reads the colour-(1-c) bits the other ranges just
    // wrote); every thread of the block passes the barriers
#pragma unroll 1
    for (int t = 0; t < theta; ++t) {
      const uint32_t T = T0 + (uint32_t)t;
      hs.key = sweep_key((uint32_t)slot, T, rk);
#pragma unroll 1
      for (uint32_t c = 0; c < 2; ++c) {
        hs.c = c;
        hs.half = build_half_table<GEO, TPB, P>(s_tab, 2 * t + (int)c, c, T) + part;
        if (live) half_sweep3d<GEO, CS, RPP>(col, s_bond, hs, rk, y0);
      }
    }
  } else {
    // one thread per replica: the 2 theta half sweeps in chunks of NH tables,
    // one block barrier per chunk
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
          if (c == 0) hs.key = sweep_key((uint32_t)slot, T0 + (uint32_t)((h0 + j) >> 1), rk);
          hs.c = c;
          hs.half = half_table<GEO, P>(s_tab, j);
          half_sweep3d<GEO, CS, RPP>(col, s_bond, hs, rk, y0);
        }
      }
    }
  }
  __syncthreads();  // every row range swept before the energy reads its neighbour rows
  int E = 0;
  if (live) {
    int sat = satisfied_rows<GEO, CS>(col, s_bond, y0, y0 + RPP);
#pragma unroll
    for (int off = RW; off < 32; off <<= 1) sat += __shfl_xor_sync(hs.lanes, sat, off);
    E = GEO::NB - 2 * sat;
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
  measure_store(R, nxt, slot, live && part == 0, E);
}

// Sec. 2: R0 independent uniformly random microstates at beta = 0.  Word w of
// slot s is word (w mod 4) of Philox(ctr = (w div 4, s, 0, TAG_INIT)),
// restricted to the valid lanes.
template <int L, int TPB>
__global__ void __launch_bounds__(TPB) k_init3d(RunDev* __restrict__ runs, const Work* __restrict__ table) {
  using GEO = Geo3<L>;
  constexpr int WR = GEO::WR, W = GEO::W;
  extern __shared__ uint32_t smem[];
  uint32_t* s_bond = smem;
  uint32_t* s_spin = smem + 6 * W;
  const Work wk = table[blockIdx.x];
  RunDev& R = runs[wk.run];
  const int64_t R0 = R.R;
  if ((int64_t)wk.first >= R0) return;
  const int tid = threadIdx.x;
  for (int i = tid; i < 6 * W; i += TPB) s_bond[i] = R.bonds[i];
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
    E = GEO::NB - 2 * satisfied_rows<GEO, TPB>(col, s_bond, 0, L);
    store_column<GEO, TPB>(R.spins[0] + (size_t)slot * W, col);
  }
  measure_store(R, 0, slot, live, E);
}

template <int L, int TPB>
inline size_t init3d_smem() {
  using GEO = Geo3<L>;
  return sizeof(uint32_t) * (6 * GEO::W + GEO::WR * TPB);
}

// One launch over nwork work items (TPB slots each); the dynamic shared
// memory limit is raised where the kernel needs more than 48 KiB (also when
// nwork is 0, so that it can be set outside a stream capture).
template <int L, int TPB, int P>
cudaError_t launch_sweep3d_p(RunDev* runs, const Work* table, int nwork, cudaStream_t st) {
  if constexpr (!split_ok<Geo3<L>>(P) || TPB / P < 4 || (P > 1 && TPB < 64)) {
    return cudaErrorInvalidValue;
  } else {
    const size_t sm = sizeof(uint32_t) * SweepShape<L, TPB, P>::SMEM_WORDS;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute((const void*)k_sweep3d<L, TPB, P>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    if (nwork <= 0) return cudaSuccess;
    k_sweep3d<L, TPB, P><<<nwork * P, TPB, sm, st>>>(runs, table);
    return cudaGetLastError();
  }
}

template <int L, int TPB>
cudaError_t launch_sweep3d_t(RunDev* runs, const Work* table, int nwork, cudaStream_t st, bool init, int split) {
  if (init) {
    const size_t sm = init3d_smem<L, TPB>();
    if (sm > 48 * 1024) {
      cudaError_t e =
          cudaFuncSetAttribute((const void*)k_init3d<L, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    if (nwork <= 0) return cudaSuccess;
    k_init3d<L, TPB><<<nwork, TPB, sm, st>>>(runs, table);
    return cudaGetLastError();
  }
  switch (split) {
    case 1: return launch_sweep3d_p<L, TPB, 1>(runs, table, nwork, st);
    case 2: return launch_sweep3d_p<L, TPB, 2>(runs, table, nwork, st);
    case 4: return launch_sweep3d_p<L, TPB, 4>(runs, table, nwork, st);
    case 8: return launch_sweep3d_p<L, TPB, 8>(runs, table, nwork, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pa

// Threads per replica the sweep kernel supports for edge L (1, 2, 4, 8).
#define PA_INSTANTIATE_SWEEP3D(LL)                                                                        \
  namespace pa {                                                                                          \
  cudaError_t launch_sweep3d_L##LL(int tpb, int split, RunDev* runs, const Work* table, int nwork,       \
                                   cudaStream_t st, bool init) {                                          \
    switch (tpb) {                                                                                        \
      case 32: return launch_sweep3d_t<LL, 32>(runs, table, nwork, st, init, split);                      \
      case 64: return launch_sweep3d_t<LL, 64>(runs, table, nwork, st, init, split);                      \
      case 128: return launch_sweep3d_t<LL, 128>(runs, table, nwork, st, init, split);                    \
      case 256: return launch_sweep3d_t<LL, 256>(runs, table, nwork, st, init, split);                    \
      default: return cudaErrorInvalidValue;                                                              \
    }                                                                                                     \
  }                                                                                                       \
  bool sweep3d_split_ok_L##LL(int split) { return split_ok<Geo3<LL>>(split); }                            \
  }
