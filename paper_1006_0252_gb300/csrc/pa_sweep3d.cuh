// pa_sweep3d.cuh -- fused replica copy + checkerboard Metropolis sweeps +
// energy measurement for 3D periodic cubic +-1 spin glasses (Sec. 2: "all
// replicas are now subject to an equilibrating MCMC process at the new
// temperature"; Algorithm: "Equilibrate replica j for theta sweeps", then
// "Compute observables").
//
// One thread owns one replica.  Its packed words live in a column of shared
// memory (word w of thread t at s_spin[w * TPB + t], so a warp touches 32
// consecutive banks); a half-sweep walks the y-rows with a three-row sliding
// window in registers and updates the G words of a row with 32-bit bitwise
// logic: for every direction d the bond bit b_d = s ^ s_nb ^ j_d is 1 where
// the bond is satisfied (J s s' = -1), a carry-save adder counts the n
// satisfied bonds per site (dE = 4n - 12), and a site flips iff n <= 3 or its
// uniform u < threshold[dE/2] (only energy rises draw on the uniform).
#pragma once
#include <type_traits>
#include "pa_device.cuh"

namespace pa {

// Bond masks of one run: [6][W] words; direction order x+, x-, y+, y-, z+, z-;
// bit (w, p) set iff the coupling of that bond of site (w, p) is -1.
enum { DXP = 0, DXM = 1, DYP = 2, DYM = 3, DZP = 4, DZM = 5 };

template <class GEO>
__device__ __forceinline__ uint32_t rot_xp(uint32_t s) {  // neighbour x+1 within each lane
  return ((s >> 1) & ~GEO::HI) | ((s << (GEO::L - 1)) & GEO::HI);
}
template <class GEO>
__device__ __forceinline__ uint32_t rot_xm(uint32_t s) {  // neighbour x-1 within each lane
  return ((s << 1) & ~GEO::LO) | ((s >> (GEO::L - 1)) & GEO::LO);
}
template <class GEO>
__device__ __forceinline__ uint32_t lanes_down(uint32_t s) {  // lane j <- lane j+1 (z+1 across g wrap)
  if constexpr (GEO::K == 1) {
    return s;
  } else {
    return (s >> GEO::L) | (s << (GEO::L * (GEO::K - 1)));
  }
}
template <class GEO>
__device__ __forceinline__ uint32_t lanes_up(uint32_t s) {  // lane j <- lane j-1 (z-1 across g wrap)
  if constexpr (GEO::K == 1) {
    return s;
  } else {
    return (s << GEO::L) | ((s & GEO::VALID) >> (GEO::L * (GEO::K - 1)));
  }
}

// Satisfied-bond counts of the "+" bonds of one word (energy measurement).
template <class GEO>
__device__ __forceinline__ int plus_bonds_satisfied(uint32_t s, uint32_t yp, uint32_t zp,
                                                    uint32_t jxp, uint32_t jyp, uint32_t jzp) {
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
      sat += plus_bonds_satisfied<GEO>(row[g], rowp[g], zp, s_bond[DXP * W + w],
                                       s_bond[DYP * W + w], s_bond[DZP * W + w]);
    }
  }
  return sat;
}

// Energy of the replica in this thread's shared-memory column.
template <class GEO, int TPB>
__device__ __forceinline__ int energy3d(const uint32_t* __restrict__ col,
                                        const uint32_t* __restrict__ s_bond) {
  return GEO::NB - 2 * satisfied_rows<GEO, TPB>(col, s_bond, 0, GEO::L);
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

template <class GEO, int TPB>
__device__ __forceinline__ void store_column(uint32_t* __restrict__ dst, const uint32_t* __restrict__ col) {
  constexpr int WR = GEO::WR, W = GEO::W;
  uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll 4
  for (int q = 0; q < W / 4; ++q) {
    uint4 v;
    v.x = (4 * q + 0 < WR) ? col[(4 * q + 0) * TPB] : 0u;
    v.y = (4 * q + 1 < WR) ? col[(4 * q + 1) * TPB] : 0u;
    v.z = (4 * q + 2 < WR) ? col[(4 * q + 2) * TPB] : 0u;
    v.w = (4 * q + 3 < WR) ? col[(4 * q + 3) * TPB] : 0u;
    d4[q] = v;
  }
}

// Which threshold compares run on the multiply-add pipe instead of the
// integer ALU pipe (the ALU pipe is the sweep kernel's bottleneck).
#ifndef PA_SWEEP_CMP_MODE
#define PA_SWEEP_CMP_MODE 0
#endif
constexpr bool CMP_FMA4 = PA_SWEEP_CMP_MODE >= 2;
constexpr bool CMP_FMA8 = PA_SWEEP_CMP_MODE >= 1;
constexpr bool CMP_FMA12 = PA_SWEEP_CMP_MODE >= 1;

// Bit 2m set iff u[m] < thr, for m < SITES.  ON_FMA: the compare is the
// high word of u*one + (2^32 - thr) (= [u >= thr], one == 1 at run time) and
// the bits are gathered by mask = mask*4 + hi, both multiply-adds; the
// result is complemented onto the even positions at the end.
template <int SITES, bool ON_FMA, int OFF = 0>
__device__ __forceinline__ uint32_t lt_mask(const uint32_t* u, uint32_t thr, uint64_t cthr, uint32_t one) {
  u += OFF;
  if constexpr (ON_FMA) {
    const uint32_t four = one << 2;
    uint32_t ge = 0u;
#pragma unroll
    for (int m = SITES - 1; m >= 0; --m) {
      uint64_t r;
      asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(u[m]), "r"(one), "l"(cthr));
      const uint32_t hi = (uint32_t)(r >> 32);
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(ge) : "r"(ge), "r"(four), "r"(hi));
    }
    constexpr uint32_t EV = (2 * SITES >= 32) ? 0x55555555u : (0x55555555u & ((1u << (2 * SITES)) - 1u));
    return EV & ~ge;
  } else {
    uint32_t lt = 0u;
#pragma unroll
    for (int m = 0; m < SITES; ++m) lt |= (u[m] < thr) ? (1u << (2 * m)) : 0u;
    return lt;
  }
}

// Uniforms of the colour-c sites of one word and their compares with the
// thresholds of dE = 4, 8, 12 (masks at even positions 2m: bit set iff
// u_m < thr).  The word's first site has colour-c rank r0 = w SITES, so its
// uniforms are words A .. A + SITES - 1 (A = r0 mod 4) of the Philox calls
// q0 = r0 div 4, q0 + 1, ...; a call shared with the previous word (A > 0)
// is taken from `carry`, and a call the next word shares is left there.
// thr4 >= thr8 >= thr12, so where u >= thr4 the other two compares fail as
// well: they are skipped for the word when no lane of the warp has a uniform
// below thr4 (warp-uniform branch; most words at low temperature).
template <int SITES, int A>
constexpr int word_calls() { return (A + SITES + 3) / 4; }

// The uniforms of one word (see word_compares): words A .. A + SITES - 1 of u.
template <int SITES, int A>
__device__ __forceinline__ void word_uniforms(uint32_t q0, uint32_t slot, uint32_t T, uint32_t tag,
                                              const RoundKeys& rk, uint32_t (&carry)[4],
                                              uint32_t (&u)[4 * word_calls<SITES, A>()]) {
  constexpr int NQ = word_calls<SITES, A>();
  if constexpr (A != 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = carry[i];
  }
#pragma unroll
  for (int q = (A != 0 ? 1 : 0); q < NQ; ++q) {
    const u32x4 v = philox10_rk(q0 + q, slot, T, tag, rk);
    u[4 * q + 0] = v.a;
    u[4 * q + 1] = v.b;
    u[4 * q + 2] = v.c;
    u[4 * q + 3] = v.d;
  }
  if constexpr ((A + SITES) % 4 != 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) carry[i] = u[4 * (NQ - 1) + i];
  }
}

template <int SITES, int A>
__device__ __forceinline__ void word_compares(uint32_t q0, uint32_t slot, uint32_t T, uint32_t tag,
                                              const RoundKeys& rk, uint32_t T4, uint32_t T8, uint32_t T12,
                                              uint64_t c4, uint64_t c8, uint64_t c12, uint32_t one, unsigned lanes,
                                              uint32_t (&carry)[4], uint32_t& e4, uint32_t& e8, uint32_t& e12) {
  uint32_t u[4 * word_calls<SITES, A>()];
  word_uniforms<SITES, A>(q0, slot, T, tag, rk, carry, u);
  e4 = lt_mask<SITES, CMP_FMA4, A>(u, T4, c4, one);
  e8 = 0u;
  e12 = 0u;
  if (__any_sync(lanes, e4 != 0u)) {
    e8 = lt_mask<SITES, CMP_FMA8, A>(u, T8, c8, one);
    if (__any_sync(lanes, e8 != 0u)) e12 = lt_mask<SITES, CMP_FMA12, A>(u, T12, c12, one);
  }
}

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// Word g of row y: bond bits, satisfied-bond count, compares, flips.  A is
// the alignment of the word's first uniform (see word_compares).
template <class GEO, int TPB, int A>
__device__ __forceinline__ void word3d(int g, int y, const uint32_t* __restrict__ s_bond, uint32_t (&rowm)[GEO::G],
                                       uint32_t (&row)[GEO::G], const uint32_t (&rowp)[GEO::G], uint32_t slot,
                                       uint32_t T, uint32_t c, uint32_t tag, const RoundKeys& rk, uint32_t T4,
                                       uint32_t T8, uint32_t T12, uint64_t c4, uint64_t c8, uint64_t c12,
                                       uint32_t one, unsigned lanes, uint32_t (&carry)[4]) {
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
  // uniforms of the colour-c sites of this word, compared with the
  // thresholds of dE = 4, 8, 12 (n = 4, 5, 6)
  uint32_t e4, e8, e12;
  word_compares<SITES, A>((uint32_t)(w * SITES) >> 2, slot, T, tag, rk, T4, T8, T12, c4, c8, c12, one, lanes, carry,
                          e4, e8, e12);
  const uint32_t par0 = (c + (uint32_t)y + (uint32_t)g) & 1u;
  const uint32_t cm = to_colour_positions<GEO>(GEO::EVEN, par0);
  const uint32_t a4 = to_colour_positions<GEO>(e4, par0);
  const uint32_t a8 = to_colour_positions<GEO>(e8, par0);
  const uint32_t a12 = to_colour_positions<GEO>(e12, par0);
  const uint32_t sel = (n1 & a12) | (~n1 & ((n0 & a8) | (~n0 & a4)));
  row[g] = s ^ (cm & (~n2 | sel));
}

// Row y of a half sweep (three-row window rowm / row / rowp).  YP is the
// row's position in its pair of rows (y mod 2 when SITES is not a multiple of
// 4): a pair of rows holds L^2/2 sites of each colour, a multiple of 4, so
// the alignment of every word's first uniform is known at compile time.
template <class GEO, int TPB, int YP>
__device__ __forceinline__ void row3d(uint32_t* __restrict__ col, const uint32_t* __restrict__ s_bond, int y,
                                      uint32_t (&rowm)[GEO::G], uint32_t (&row)[GEO::G], uint32_t (&rowp)[GEO::G],
                                      uint32_t slot, uint32_t T, uint32_t c, const RoundKeys& rk, uint32_t T4,
                                      uint32_t T8, uint32_t T12, uint64_t c4, uint64_t c8, uint64_t c12, uint32_t one,
                                      unsigned lanes, uint32_t (&carry)[4]) {
  constexpr int G = GEO::G, L = GEO::L, K = GEO::K;
  constexpr int SITES = K * L / 2;  // colour-c sites per word
  const uint32_t tag = TAG_SWEEP + c;
  const int yn = (y + 1 == L) ? 0 : y + 1;
#pragma unroll
  for (int g = 0; g < G; ++g) rowp[g] = col[(yn * G + g) * TPB];
  if constexpr (SITES % 4 == 0) {
#pragma unroll
    for (int g = 0; g < G; ++g)
      word3d<GEO, TPB, 0>(g, y, s_bond, rowm, row, rowp, slot, T, c, tag, rk, T4, T8, T12, c4, c8, c12, one, lanes,
                          carry);
  } else {
    static_for<0, G>([&](auto gc) {
      constexpr int g = decltype(gc)::value;
      constexpr int A = (SITES * (YP * G + g)) % 4;
      word3d<GEO, TPB, A>(g, y, s_bond, rowm, row, rowp, slot, T, c, tag, rk, T4, T8, T12, c4, c8, c12, one, lanes,
                          carry);
    });
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    col[(y * G + g) * TPB] = row[g];
    rowm[g] = row[g];
    row[g] = rowp[g];
  }
}

// One Metropolis half-sweep over the colour-c sites of rows y0 .. y1-1 of
// one replica (the whole replica: 0 .. L).  Colour-c sites only read
// colour-(1-c) neighbours, which a half sweep does not change, so disjoint
// row ranges of one replica may be swept by different threads at once; for
// SITES not a multiple of 4, y0 and y1 must be even (whole pairs of rows).
template <class GEO, int TPB>
__device__ __forceinline__ void half_sweep3d(uint32_t* __restrict__ col,
                                             const uint32_t* __restrict__ s_bond, uint32_t slot,
                                             uint32_t T, uint32_t c, const RoundKeys& rk,
                                             uint32_t T4, uint32_t T8, uint32_t T12,
                                             uint64_t c4, uint64_t c8, uint64_t c12, uint32_t one,
                                             unsigned lanes, int y0 = 0, int y1 = GEO::L) {
  constexpr int G = GEO::G, L = GEO::L, K = GEO::K;
  constexpr int SITES = K * L / 2;  // colour-c sites per word
  uint32_t rowm[G], row[G], rowp[G];
  uint32_t carry[4] = {0u, 0u, 0u, 0u};
  const int ym = (y0 == 0) ? L - 1 : y0 - 1;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    rowm[g] = col[(ym * G + g) * TPB];
    row[g] = col[(y0 * G + g) * TPB];
  }
  if constexpr (SITES % 4 == 0) {
#pragma unroll 1
    for (int y = y0; y < y1; ++y)
      row3d<GEO, TPB, 0>(col, s_bond, y, rowm, row, rowp, slot, T, c, rk, T4, T8, T12, c4, c8, c12, one, lanes,
                         carry);
  } else {
#pragma unroll 1
    for (int y = y0; y < y1; y += 2) {
      row3d<GEO, TPB, 0>(col, s_bond, y, rowm, row, rowp, slot, T, c, rk, T4, T8, T12, c4, c8, c12, one, lanes,
                         carry);
      row3d<GEO, TPB, 1>(col, s_bond, y + 1, rowm, row, rowp, slot, T, c, rk, T4, T8, T12, c4, c8, c12, one,
                         lanes, carry);
    }
  }
}

// Wave tail.  A thread holds one replica for the whole step, so when the
// population exceeds a whole number of waves of resident threads by a few
// replicas, those few run as a nearly empty last wave at the speed of one
// replica.  Such a tail is swept by SPLIT_P threads per replica instead, each
// taking L / SPLIT_P consecutive rows.  This needs colour-c sites per word a
// multiple of 4 (no uniform shared between rows of different threads) and is
// compiled for L = 8 and 12 only: for L = 4 the tail path would cost the
// kernel a warp per sub-partition, for L = 16 register spills.  The P threads
// of a replica are lanes l, l + 32/P, ... of one warp and meet at __syncwarp
// after every half sweep.
template <class GEO>
constexpr int split_parts() {
  return ((GEO::K * GEO::L / 2) % 4 == 0 && (GEO::L == 8 || GEO::L == 12)) ? 4 : 1;
}

// Column stride of a tail block: NR replicas per block, the P threads of a
// replica reading rows D words apart; a stride with D * stride = (32 / P) u
// (mod 32), u odd, puts the P threads on different banks.
constexpr int split_stride(int NR, int D, int P, int TPB) {
  for (int cs = NR; cs < NR + 32 && cs <= TPB; ++cs) {
    const int m = (D * cs) % 32;
    if (m % (32 / P) == 0 && ((m / (32 / P)) & 1)) return cs;
  }
  return NR;
}

template <class GEO, int TPB>
__device__ __forceinline__ void sweep3d_split(RunDev& R, uint32_t* __restrict__ s_spin,
                                              const uint32_t* __restrict__ s_bond, int64_t first, int64_t Rn) {
  constexpr int P = split_parts<GEO>();
  constexpr int WR = GEO::WR, W = GEO::W, L = GEO::L, G = GEO::G;
  constexpr int RW = 32 / P;       // replicas per warp
  constexpr int NR = TPB / P;      // replicas per block
  constexpr int RPP = L / P;       // rows per thread
  constexpr int CS = split_stride(NR, RPP * G, P, TPB);
  const int tid = threadIdx.x, lane = tid & 31;
  const int r = (tid >> 5) * RW + (lane % RW);
  const int part = lane / RW;
  const int64_t slot = first + r;
  const bool live = slot < Rn;
  const int cur = R.cur, nxt = cur ^ 1;
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
  const unsigned lanes = __ballot_sync(0xFFFFFFFFu, live);
  int E = 0;
  if (live) {
    const RoundKeys rk = make_round_keys(R.seed);
    const uint32_t T4 = R.thr[2], T8 = R.thr[4], T12 = R.thr[6];
    const uint64_t c4 = (1ull << 32) - T4, c8 = (1ull << 32) - T8, c12 = (1ull << 32) - T12;
    const uint32_t one = R.one;
    const int theta = R.theta_next;
    const uint32_t T0 = (uint32_t)R.sweeps;
    const int y0 = part * RPP;
#pragma unroll 1
    for (int t = 0; t < theta; ++t) {
#pragma unroll 1
      for (uint32_t c = 0; c < 2; ++c) {
        half_sweep3d<GEO, CS>(col, s_bond, (uint32_t)slot, T0 + (uint32_t)t, c, rk, T4, T8, T12, c4, c8, c12,
                              one, lanes, y0, y0 + RPP);
        __syncwarp(lanes);
      }
    }
    int sat = satisfied_rows<GEO, CS>(col, s_bond, y0, y0 + RPP);
#pragma unroll
    for (int off = RW; off < 32; off <<= 1) sat += __shfl_xor_sync(lanes, sat, off);
    E = GEO::NB - 2 * sat;
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
  measure_store(R, nxt, slot, live && part == 0, E);
}

// Blocks 0 .. nmain-1 take the work table (one thread per replica); for a
// class with one run and wave > 0 (the replicas one launch holds resident),
// blocks nmain .. are tail blocks: when R~' exceeds a whole number of waves by
// at most wave / SPLIT_P replicas, those replicas are swept SPLIT_P threads
// each by the tail blocks instead (see sweep3d_split).  The keying of every
// uniform is the replica's and the word's, so both ways give the same bits.
template <int L, int TPB>
__global__ void __launch_bounds__(TPB) k_sweep3d(RunDev* __restrict__ runs,
                                                 const Work* __restrict__ table, int nmain, int64_t wave) {
  using GEO = Geo3<L>;
  constexpr int WR = GEO::WR, W = GEO::W;
  constexpr int P = split_parts<GEO>();
  extern __shared__ uint32_t smem[];
  uint32_t* s_bond = smem;               // [6][W]
  uint32_t* s_spin = smem + 6 * W;       // [WR][TPB]
  const bool tail = (int)blockIdx.x >= nmain;
  const Work wk = table[tail ? 0 : blockIdx.x];
  RunDev& R = runs[wk.run];
  if (R.skip) return;
  const int64_t Rn = R.R_next;
  int64_t main_end = Rn;
  if (P > 1 && wave > 0) {
    const int64_t nfull = Rn / wave, rest = Rn - nfull * wave;
    if (nfull >= 1 && rest > 0 && rest * P <= wave) main_end = nfull * wave;
  }
  const int tid = threadIdx.x;
  if constexpr (P > 1) {
    if (tail) {
      const int64_t first = main_end + (int64_t)((int)blockIdx.x - nmain) * (TPB / P);
      if (main_end == Rn || first >= Rn) return;
      for (int i = tid; i < 6 * W; i += TPB) s_bond[i] = R.bonds[i];
      sweep3d_split<GEO, TPB>(R, s_spin, s_bond, first, Rn);
      return;
    }
  }
  if ((int64_t)wk.first >= main_end) return;
  for (int i = tid; i < 6 * W; i += TPB) s_bond[i] = R.bonds[i];
  const int64_t slot = (int64_t)wk.first + tid;
  const bool live = slot < main_end;
  const int cur = R.cur, nxt = cur ^ 1;
  uint32_t* col = s_spin + tid;
  if (live) {
    const int32_t src = R.src[slot];
    const uint4* p4 = reinterpret_cast<const uint4*>(R.spins[cur] + (size_t)src * W);
#pragma unroll 4
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
    const uint32_t T4 = R.thr[2], T8 = R.thr[4], T12 = R.thr[6];
    const uint64_t c4 = (1ull << 32) - T4, c8 = (1ull << 32) - T8, c12 = (1ull << 32) - T12;
    const uint32_t one = R.one;
    const int theta = R.theta_next;
    const uint32_t T0 = (uint32_t)R.sweeps;
#pragma unroll 1
    for (int t = 0; t < theta; ++t) {
#pragma unroll 1
      for (uint32_t c = 0; c < 2; ++c)
        half_sweep3d<GEO, TPB>(col, s_bond, (uint32_t)slot, T0 + (uint32_t)t, c, rk, T4, T8, T12, c4, c8,
                               c12, one, lanes);
    }
    E = energy3d<GEO, TPB>(col, s_bond);
    store_column<GEO, TPB>(R.spins[nxt] + (size_t)slot * W, col);
  }
  measure_store(R, nxt, slot, live, E);
}

// Sec. 2: R0 independent uniformly random microstates at beta = 0.  Word w of
// slot s is word (w mod 4) of Philox(ctr = (w div 4, s, 0, TAG_INIT)),
// restricted to the valid lanes.
template <int L, int TPB>
__global__ void __launch_bounds__(TPB) k_init3d(RunDev* __restrict__ runs,
                                                const Work* __restrict__ table) {
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
    E = energy3d<GEO, TPB>(col, s_bond);
    store_column<GEO, TPB>(R.spins[0] + (size_t)slot * W, col);
  }
  measure_store(R, 0, slot, live, E);
}

template <int L, int TPB>
inline size_t sweep3d_smem() {
  using GEO = Geo3<L>;
  return sizeof(uint32_t) * (6 * GEO::W + GEO::WR * TPB);
}

// wave > 0: the launch sweeps one run, wave = replicas resident at once
// (sweep3d_wave); tail blocks are appended for the split of a wave tail.
template <int L, int TPB>
cudaError_t launch_sweep3d_t(RunDev* runs, const Work* table, int nwork, cudaStream_t st,
                             bool init, int64_t wave) {
  const size_t sm = sweep3d_smem<L, TPB>();
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(init ? (const void*)k_init3d<L, TPB> : (const void*)k_sweep3d<L, TPB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (nwork <= 0) return cudaSuccess;
  if (init) {
    k_init3d<L, TPB><<<nwork, TPB, sm, st>>>(runs, table);
  } else {
    constexpr int P = split_parts<Geo3<L>>();
    const int ntail = (P > 1 && wave > 0) ? (int)((wave + TPB - 1) / TPB) : 0;
    k_sweep3d<L, TPB><<<nwork + ntail, TPB, sm, st>>>(runs, table, nwork, P > 1 ? wave : 0);
  }
  return cudaGetLastError();
}

// Replicas one launch of the sweep kernel holds resident on the device.
template <int L, int TPB>
int64_t sweep3d_wave_t() {
  int dev = 0, nsm = 0, nb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const size_t sm = sweep3d_smem<L, TPB>();
  if (sm > 48 * 1024 &&
      cudaFuncSetAttribute(k_sweep3d<L, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep3d<L, TPB>, TPB, sm) != cudaSuccess) return 0;
  return (int64_t)nb * nsm * TPB;
}

}  // namespace pa

#define PA_INSTANTIATE_SWEEP3D(LL)                                                          \
  namespace pa {                                                                            \
  cudaError_t launch_sweep3d_L##LL(int tpb, RunDev* runs, const Work* table, int nwork,     \
                                   cudaStream_t st, bool init, int64_t wave) {              \
    switch (tpb) {                                                                          \
      case 32: return launch_sweep3d_t<LL, 32>(runs, table, nwork, st, init, wave);         \
      case 64: return launch_sweep3d_t<LL, 64>(runs, table, nwork, st, init, wave);         \
      case 128: return launch_sweep3d_t<LL, 128>(runs, table, nwork, st, init, wave);       \
      case 256: return launch_sweep3d_t<LL, 256>(runs, table, nwork, st, init, wave);       \
      default: return cudaErrorInvalidValue;                                                \
    }                                                                                       \
  }                                                                                         \
  int64_t sweep3d_wave_L##LL(int tpb) {                                                     \
    switch (tpb) {                                                                          \
      case 32: return sweep3d_wave_t<LL, 32>();                                             \
      case 64: return sweep3d_wave_t<LL, 64>();                                             \
      case 128: return sweep3d_wave_t<LL, 128>();                                           \
      case 256: return sweep3d_wave_t<LL, 256>();                                           \
      default: return 0;                                                                    \
    }                                                                                       \
  }                                                                                         \
  }
