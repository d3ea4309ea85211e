// pa_lattice3d.cuh -- pieces shared by the 3D sweep kernels (+-1 and Gaussian
// couplings): neighbour words of the packed lattice, the column layout of a
// replica in shared memory, and the sweep uniforms.
//
// Sweep uniforms.  The colour-c site of rank r in slot s at global sweep T
// uses word r mod 4 of Philox4x32-10 at counter (q, s, T, TAG_SWEEP + c),
// q = r div 4.  Round 0 multiplies the counter words c0 = q and c2 = T, round
// 1 the words a0 (a function of s and T only) and a2 (a function of q and c
// only).  So:
//   * the products of q and of a2 are the same for every slot and sweep: they
//     are tabulated once per launch, per colour and call index q (CallEntry);
//   * the products of T and of a0 are the same for every call of one half
//     sweep of one slot: they are computed once per half sweep (SweepKey);
//   * round 2 multiplies b0 (a function of q, c and T: the same for every
//     slot) and b2 (per slot and call); b0's product is tabulated once per
//     half sweep for the whole block (HalfEntry).
// Each call then starts at round 2 with one 32x32->64 multiply instead of six
// in rounds 0-2; rounds 3-9 are the generator's as they stand.  The state
// entering round 3 is the state the plain generator reaches, word for word,
// so the uniforms are bit-identical to philox10(q, s, T, TAG_SWEEP + c).
#pragma once
#include <type_traits>
#include "pa_device.cuh"

namespace pa {

// ---------------------------------------------------------------------------
// Neighbour words (see Geo3 in pa_device.cuh for the packing).
// ---------------------------------------------------------------------------
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

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// Write a replica's column (word w at col[w * CS]) to its global row, 16
// bytes at a time; words WR .. W-1 of the row are zero padding.
template <class GEO, int CS>
__device__ __forceinline__ void store_column(uint32_t* __restrict__ dst, const uint32_t* __restrict__ col) {
  constexpr int WR = GEO::WR, W = GEO::W;
  uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll 4
  for (int q = 0; q < W / 4; ++q) {
    uint4 v;
    v.x = (4 * q + 0 < WR) ? col[(4 * q + 0) * CS] : 0u;
    v.y = (4 * q + 1 < WR) ? col[(4 * q + 1) * CS] : 0u;
    v.z = (4 * q + 2 < WR) ? col[(4 * q + 2) * CS] : 0u;
    v.w = (4 * q + 3 < WR) ? col[(4 * q + 3) * CS] : 0u;
    d4[q] = v;
  }
}

// ---------------------------------------------------------------------------
// P threads per replica.  A replica's rows are split into P ranges of L / P
// consecutive y-rows, one per thread; colour-c sites read only colour-(1-c)
// neighbours, which a half sweep leaves unchanged, so the P ranges are swept
// at once and meet at a barrier after every half sweep.  Where the colour-c
// sites of a word are not a multiple of 4 a Philox call is shared by two
// consecutive rows, so a range must hold whole pairs of rows.  The P threads
// of a replica are lanes l, l + 32/P, ... of one warp.
// ---------------------------------------------------------------------------
template <class GEO>
constexpr bool split_ok(int P) {
  if (P != 1 && P != 2 && P != 4 && P != 8) return false;
  if (GEO::L % P != 0) return false;
  if (P == 1) return true;
  return ((GEO::L / P) % 2 == 0) || ((GEO::K * GEO::L / 2) % 4 == 0);
}

// Column stride of a block of NR replicas whose P threads read rows D words
// apart: a stride with D * stride = (32 / P) u (mod 32), u odd, puts the P
// threads of a replica on different banks (NR itself when P = 1).
constexpr int split_stride(int NR, int D, int P, int TPB) {
  for (int cs = NR; cs < NR + 32 && cs <= TPB; ++cs) {
    const int m = (D * cs) % 32;
    if (m % (32 / P) == 0 && ((m / (32 / P)) & 1)) return cs;
  }
  return NR;
}

// ---------------------------------------------------------------------------
// Sweep uniforms from tables (see the file comment).
// ---------------------------------------------------------------------------
struct SweepKey {
  uint32_t A1;   // lo(M1 T): counter word 1 after round 0
  uint32_t H;    // hi(M0 a0), a0 = hi(M1 T) ^ s ^ k0[0]
  uint32_t B3x;  // lo(M0 a0) ^ k1[2]: word 3 after round 1, with round 2's key
};

__device__ __forceinline__ SweepKey sweep_key(uint32_t slot, uint32_t T, const RoundKeys& rk) {
  SweepKey k;
  k.A1 = PHILOX_MUL1 * T;
  const uint32_t a0 = __umulhi(PHILOX_MUL1, T) ^ slot ^ rk.k0[0];
  k.H = __umulhi(PHILOX_MUL0, a0);
  k.B3x = (PHILOX_MUL0 * a0) ^ rk.k1[2];
  return k;
}

// Call entry of call q, tag TAG_SWEEP + c: {x, y, z, 0} with
// x = lo(M0 q) ^ k1[1], y = hi(M1 a2) ^ k0[1], z = lo(M1 a2) ^ k0[2],
// a2 = hi(M0 q) ^ tag ^ k1[0].
__device__ __forceinline__ uint4 sweep_call_entry(uint32_t q, uint32_t tag, const RoundKeys& rk) {
  const uint32_t a2 = __umulhi(PHILOX_MUL0, q) ^ tag ^ rk.k1[0];
  uint4 e;
  e.x = (PHILOX_MUL0 * q) ^ rk.k1[1];
  e.y = __umulhi(PHILOX_MUL1, a2) ^ rk.k0[1];
  e.z = (PHILOX_MUL1 * a2) ^ rk.k0[2];
  e.w = 0u;
  return e;
}

// Half-sweep entry from a call entry at sweep T: {x, z, hi(M0 b0), lo(M0 b0)},
// b0 = y ^ lo(M1 T) = hi(M1 a2) ^ a1 ^ k0[1] (word 0 after round 1).
__device__ __forceinline__ uint4 sweep_half_entry(const uint4& e, uint32_t A1) {
  const uint32_t b0 = e.y ^ A1;
  uint4 h;
  h.x = e.x;
  h.y = e.z;
  h.z = __umulhi(PHILOX_MUL0, b0);
  h.w = PHILOX_MUL0 * b0;
  return h;
}

// The four uniforms of one call: round 2 from the half-sweep entry and the
// slot's key, then rounds 3-9.
__device__ __forceinline__ u32x4 philox_sweep(const uint4& h, const SweepKey& k, const RoundKeys& rk) {
  const uint32_t b2 = k.H ^ h.x;  // word 2 after round 1
  uint32_t c0 = __umulhi(PHILOX_MUL1, b2) ^ h.y;
  uint32_t c1 = PHILOX_MUL1 * b2;
  uint32_t c2 = h.z ^ k.B3x;
  uint32_t c3 = h.w;
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(PHILOX_MUL0, c0);
    const uint32_t lo0 = PHILOX_MUL0 * c0;
    const uint32_t hi1 = __umulhi(PHILOX_MUL1, c2);
    const uint32_t lo1 = PHILOX_MUL1 * c2;
    c0 = hi1 ^ c1 ^ rk.k0[r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ rk.k1[r];
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// Calls per colour and replica: ceil((N / 2) / 4).
template <class GEO>
constexpr int calls_per_colour() {
  return (GEO::WR * (GEO::K * GEO::L / 2) + 3) / 4;
}

// Calls of one row range of P: (L / P) rows x G words x (SITES / 4) calls.
// The P ranges of a replica read their half-sweep entries at the same time;
// one padding entry after every range puts those reads on different banks.
template <class GEO, int P>
constexpr int calls_per_range() {
  return P == 1 ? calls_per_colour<GEO>() : (GEO::L / P) * GEO::G * (GEO::K * GEO::L / 2) / 4;
}
template <class GEO, int P>
constexpr int half_buffer_entries() {
  return calls_per_colour<GEO>() + calls_per_colour<GEO>() / calls_per_range<GEO, P>() + 1;
}

// Half-sweep tables a block of TPB threads holds at once: an even number
// from 2 to 20, as many as fit, next to the block's other `other_bytes` of
// shared memory, in about 216 bytes per thread of the block (so that the
// tables do not lower the occupancy the registers allow).  The block builds
// the tables of that many half sweeps behind one barrier; between the half
// sweeps of a chunk only the P threads of a replica (lanes of one warp)
// synchronise.
template <class GEO, int TPB, int P>
constexpr int half_tables(int other_bytes) {
  const int room = 216 * TPB - 32 * calls_per_colour<GEO>() - other_bytes;
  const int n = room > 0 ? room / (16 * half_buffer_entries<GEO, P>()) : 0;
  return n >= 20 ? 20 : (n < 2 ? 2 : (n & ~1));
}

// Shared-memory words of the tables: call entries [2 colours][Q] and NH
// padded half-sweep tables [NH][Q + Q / S + 1], all uint4.
template <class GEO, int P>
constexpr int sweep_table_words(int NH) {
  return 8 * calls_per_colour<GEO>() + 4 * NH * half_buffer_entries<GEO, P>();
}

// Call entries of both colours (all threads of the block; a barrier must
// follow before the first half-sweep table is built from them).
template <class GEO, int TPB>
__device__ __forceinline__ void fill_call_table(uint4* __restrict__ tab, const RoundKeys& rk) {
  constexpr int Q = calls_per_colour<GEO>();
  for (int i = threadIdx.x; i < 2 * Q; i += TPB) {
    const int c = i / Q, q = i - c * Q;
    tab[i] = sweep_call_entry((uint32_t)q, TAG_SWEEP + (uint32_t)c, rk);
  }
}

// Tables of half sweeps h0 .. h0 + nh - 1 (half sweep h = 2t + c is colour c
// of sweep T0 + t; h0 even, nh <= half_tables): table j at
// tab + 2Q + j (Q + Q / S + 1), entry q at q + q / S (S calls per row range).
// Every thread of the block calls this, then the block synchronises once;
// the caller synchronises the block before the next chunk overwrites them.
// The thread of row range `part` reads entry q of its range of table j at
// (half_table(tab, j) + part)[q].
template <class GEO, int P>
__device__ __forceinline__ const uint4* half_table(const uint4* tab, int j) {
  return tab + 2 * calls_per_colour<GEO>() + j * half_buffer_entries<GEO, P>();
}
// One half sweep's table, double-buffered: half sweep h = 2t + c at sweep T
// goes to table h mod 2; every thread of the block calls this, then the block
// synchronises once (a table is rewritten two half sweeps later, after the
// barrier that ends the half sweep reading it).  Returns the table.
template <class GEO, int TPB, int P>
__device__ __forceinline__ const uint4* build_half_table(uint4* __restrict__ tab, int h, uint32_t c, uint32_t T) {
  constexpr int Q = calls_per_colour<GEO>(), S = calls_per_range<GEO, P>(), HB = half_buffer_entries<GEO, P>();
  uint4* half = tab + 2 * Q + (h & 1) * HB;
  const uint32_t A1 = PHILOX_MUL1 * T;
  for (int q = threadIdx.x; q < Q; q += TPB) half[q + q / S] = sweep_half_entry(tab[c * Q + q], A1);
  __syncthreads();
  return half;
}

template <class GEO, int TPB, int P>
__device__ __forceinline__ void build_half_tables(uint4* __restrict__ tab, int h0, int nh, uint32_t T0) {
  constexpr int Q = calls_per_colour<GEO>(), S = calls_per_range<GEO, P>(), HB = half_buffer_entries<GEO, P>();
  for (int i = threadIdx.x; i < nh * Q; i += TPB) {
    const int j = i / Q, q = i - j * Q;
    const int h = h0 + j;
    const uint32_t A1 = PHILOX_MUL1 * (T0 + (uint32_t)(h >> 1));
    tab[2 * Q + j * HB + q + q / S] = sweep_half_entry(tab[(h & 1) * Q + q], A1);
  }
  __syncthreads();
}

template <int SITES, int A>
constexpr int word_calls() {
  return (A + SITES + 3) / 4;
}

// The uniforms of one word: its first colour-c site has rank r0 = w SITES, so
// they are words A .. A + SITES - 1 (A = r0 mod 4) of the calls q0 = r0 div 4,
// q0 + 1, ...; a call shared with the previous word (A > 0) is taken from
// `carry`, and a call the next word shares is left there.
template <int SITES, int A>
__device__ __forceinline__ void word_uniforms(uint32_t q0, const uint4* __restrict__ half, const SweepKey& key,
                                              const RoundKeys& rk, uint32_t (&carry)[4],
                                              uint32_t (&u)[4 * word_calls<SITES, A>()]) {
  constexpr int NQ = word_calls<SITES, A>();
  if constexpr (A != 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = carry[i];
  }
#pragma unroll
  for (int q = (A != 0 ? 1 : 0); q < NQ; ++q) {
    const u32x4 v = philox_sweep(half[q0 + q], key, rk);
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

}  // namespace pa
