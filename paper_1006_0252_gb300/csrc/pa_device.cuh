// pa_device.cuh -- device primitives of the population-annealing kernels.
//
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11),
// the uniform-double conversion and the packed-lattice geometry.  Every
// floating-point operation that decides an integer (copy counts, Metropolis
// thresholds) uses explicitly rounded intrinsics (__dmul_rn, __dadd_rn,
// __ddiv_rn, __fma_rn) so that no contraction can change a result bit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pa_internal.h"

namespace pa {

// ---------------------------------------------------------------------------
// Philox4x32-10: ten rounds of two 32x32->64 multiplies and key injection,
// the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
constexpr uint32_t PHILOX_MUL0 = 0xD2511F53u;
constexpr uint32_t PHILOX_MUL1 = 0xCD9E8D57u;
constexpr uint32_t PHILOX_BUMP0 = 0x9E3779B9u;
constexpr uint32_t PHILOX_BUMP1 = 0xBB67AE85u;

struct u32x4 {
  uint32_t a, b, c, d;
};

__device__ __forceinline__ u32x4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(PHILOX_MUL0, c0);
    const uint32_t lo0 = PHILOX_MUL0 * c0;
    const uint32_t hi1 = __umulhi(PHILOX_MUL1, c2);
    const uint32_t lo1 = PHILOX_MUL1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += PHILOX_BUMP0;
    k1 += PHILOX_BUMP1;
  }
  return {c0, c1, c2, c3};
}

// Philox with the per-round keys precomputed (rk0[r] = k0 + r*BUMP0, ...).
struct RoundKeys {
  uint32_t k0[10], k1[10];
};

__device__ __forceinline__ RoundKeys make_round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0;
    rk.k1[r] = k1;
    k0 += PHILOX_BUMP0;
    k1 += PHILOX_BUMP1;
  }
  return rk;
}

__device__ __forceinline__ u32x4 philox10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                             const RoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(PHILOX_MUL0, c0);
    const uint32_t lo0 = PHILOX_MUL0 * c0;
    const uint32_t hi1 = __umulhi(PHILOX_MUL1, c2);
    const uint32_t lo1 = PHILOX_MUL1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ rk.k0[r];
    const uint32_t n2 = hi0 ^ c3 ^ rk.k1[r];
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

__device__ __forceinline__ u32x4 philox_seeded(uint64_t seed, uint32_t c0, uint32_t c1,
                                               uint32_t c2, uint32_t c3) {
  return philox10(c0, c1, c2, c3, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t pick(const u32x4& v, int i) {
  return i == 0 ? v.a : (i == 1 ? v.b : (i == 2 ? v.c : v.d));
}

// Uniform double in [0,1) from the top 53 of the 64 bits (w0:w1).
__device__ __forceinline__ double u53(uint32_t w0, uint32_t w1) {
  const uint64_t v = ((((uint64_t)w0) << 32) | (uint64_t)w1) >> 11;
  return __dmul_rn((double)v, 0x1.0p-53);
}

// ---------------------------------------------------------------------------
// Packed-lattice geometry.
// 3D cubic edge L (even): each 32-bit word holds k lanes of L bits, k the
// largest divisor of L with k*L <= 32; G = L/k words per y-row.  Word
// w = y*G + g, lane j, bit p = j*L + x holds site (x, y, z = g + j*G).  One
// replica is L*G words, padded to a multiple of four (16-byte rows).
// 1D chain of N: bit p of word w holds site 32 w + p.
// The random-number keying refers to (w, p): sweep uniforms of the colour-c
// sites come from Philox by colour rank r = w*S + p/2 (S = K*L/2 colour-c
// sites per word, 16 in 1D): word r%4 of call r/4.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int lanes_for(int L) {
  int k = 1;
  for (int d = L; d >= 1; --d)
    if (L % d == 0 && d * L <= 32) {
      k = d;
      break;
    }
  return k;
}

template <int L_>
struct Geo3 {
  static constexpr int L = L_;
  static constexpr int K = lanes_for(L_);
  static constexpr int G = L_ / K;
  static constexpr int WR = L_ * G;
  static constexpr int W = (WR + 3) / 4 * 4;
  static constexpr int N = L_ * L_ * L_;
  static constexpr int NB = 3 * N;
  static constexpr uint32_t VALID = (K * L_ == 32) ? 0xFFFFFFFFu : ((1u << (K * L_)) - 1u);
  // bits at x = 0 / x = L-1 of every lane
  static constexpr uint32_t lane_bits(int x) {
    uint32_t m = 0;
    for (int j = 0; j < K; ++j) m |= 1u << (j * L_ + x);
    return m;
  }
  static constexpr uint32_t LO = lane_bits(0);
  static constexpr uint32_t HI = lane_bits(L_ - 1);
  // even bit positions inside the valid lanes (x even, since lanes start at
  // even positions j*L)
  static constexpr uint32_t EVEN = 0x55555555u & VALID;
  // lanes with odd j / even j
  static constexpr uint32_t lanes_parity(int par) {
    uint32_t m = 0;
    for (int j = 0; j < K; ++j)
      if ((j & 1) == par) m |= ((L_ == 32) ? 0xFFFFFFFFu : ((1u << L_) - 1u)) << (j * L_);
    return m;
  }
  static constexpr uint32_t LANES_EVEN = lanes_parity(0);
  static constexpr uint32_t LANES_ODD = lanes_parity(1);
};

// Place a mask built at even positions (one bit per colour-c site, at p = 2m)
// onto the true positions p = 2m + xpar(j), where lane j's x-parity of the
// colour-c sites is par0 ^ (j*G & 1).
template <class GEO>
__device__ __forceinline__ uint32_t to_colour_positions(uint32_t even_mask, uint32_t par0) {
  if constexpr ((GEO::G & 1) == 0) {
    return even_mask << par0;
  } else {
    return ((even_mask & GEO::LANES_EVEN) << par0) | ((even_mask & GEO::LANES_ODD) << (par0 ^ 1u));
  }
}

}  // namespace pa
