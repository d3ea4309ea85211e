// pa_box.cu -- fused replica copy + checkerboard Metropolis sweeps + energy
// measurement for general Lx x Ly x Lz boxes with any periodic/open axes
// (the 2x2x2 and 2x2x3 lattices that exact enumeration can check, Sec. 4
// nearest-neighbour bonds), for both coupling models.
//
// The packed layout and the random keying are those of the cubic kernels:
// k lanes of Lx bits per word, G = Lz / k words per y row, site (x, y, z) at
// word w = y G + (z mod G), bit p = (z div G) Lx + x.  Geometry is a run-time
// property here: for every colour-c site (word w, rank m) a shared-memory table
// holds its own bit position and those of its six neighbours (an absent bond
// points back to the site and carries J = 0), its six couplings and their sum.
// Sites of one colour only read sites of the other, so a half sweep may update
// the column in place, site by site.
#include "pa_gauss.cuh"
#include "pa_internal.h"

namespace pa {

// Largest dynamic shared memory of a block (227 KB less the static part).
constexpr size_t BOX_SMEM_MAX = 227 * 1024 - 256;

template <int TPB>
__device__ __forceinline__ uint32_t col_bit(const uint32_t* __restrict__ col, int code) {
  return (col[(code >> 5) * TPB] >> (code & 31)) & 1u;
}

// Energy E = C0 - 2 sum over "+" bonds with anti-aligned spins of J (both
// models; for +-1 couplings C0 is the sum of the couplings too).
template <int TPB>
__device__ __forceinline__ int energy_box(const uint32_t* __restrict__ col, const int32_t* __restrict__ s_code,
                                          const int32_t* __restrict__ s_J, int WR, int S, int32_t C0) {
  const int plane = WR * S;
  int32_t anti = 0;
  for (int c = 0; c < 2; ++c)
    for (int w = 0; w < WR; ++w)
      for (int m = 0; m < S; ++m) {
        const int base = w * S + m;
        const int own = s_code[(c * 7) * plane + base];
        const uint32_t so = col_bit<TPB>(col, own);
#pragma unroll
        for (int d = 0; d < 6; d += 2) {  // +x, +y, +z
          const int nb = s_code[(c * 7 + 1 + d) * plane + base];
          if (so ^ col_bit<TPB>(col, nb)) anti += s_J[(c * 6 + d) * plane + base];
        }
      }
  return C0 - 2 * anti;
}

template <int TPB>
__device__ __forceinline__ void half_sweep_box(uint32_t* __restrict__ col, const int32_t* __restrict__ s_code,
                                               const int32_t* __restrict__ s_J, const int32_t* __restrict__ s_S,
                                               int WR, int S, int model, uint32_t slot, uint32_t T,
                                               uint32_t c, const RoundKeys& rk, const uint32_t* thr, float beta_f) {
  const int plane = WR * S;
  const uint32_t tag = TAG_SWEEP + c;
  // the colour-c site of word w and rank m has colour-c rank w S + m: its
  // uniform is word (rank mod 4) of Philox call rank div 4 (one call serves
  // four consecutive ranks, across word boundaries)
  uint32_t uu[4] = {0u, 0u, 0u, 0u};
#pragma unroll 1
  for (int w = 0; w < WR; ++w) {
#pragma unroll 1
    for (int m = 0; m < S; ++m) {
      {
        const int base = w * S + m;
        const uint32_t rank = (uint32_t)base;
        if ((rank & 3u) == 0u || m == 0) {
          const u32x4 v = philox10_rk(rank >> 2, slot, T, tag, rk);
          uu[0] = v.a;
          uu[1] = v.b;
          uu[2] = v.c;
          uu[3] = v.d;
        }
        const int k = (int)(rank & 3u);
        const int own = s_code[(c * 7) * plane + base];
        const uint32_t so = col_bit<TPB>(col, own);
        int32_t acc = 0;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
          const int nb = s_code[(c * 7 + 1 + d) * plane + base];
          if (so ^ col_bit<TPB>(col, nb)) acc += s_J[(c * 6 + d) * plane + base];
        }
        const int32_t dE = 4 * acc - 2 * s_S[c * plane + base];
        bool flip;
        if (model == 1) flip = gauss_accept_fast(dE, beta_f, uu[k]);
        else flip = dE <= 0 || uu[k] < thr[dE >> 1];
        if (flip) col[(own >> 5) * TPB] ^= 1u << (own & 31);
      }
    }
  }
}

__device__ __forceinline__ void measure_box(RunDev& R, int nxt, int64_t slot, bool live, int E) {
  long long e = 0ll;
  unsigned long long lo = 0ull, hi = 0ull;
  if (live) {
    R.E[nxt][slot] = E;
    e = E;
    const unsigned long long q = (unsigned long long)((long long)E * (long long)E);
    if (R.model == 1) {
      atomicMin(&R.emin_next, (long long)E);
      lo = q & 0xFFFFFFFFull;
      hi = q >> 32;
    } else {
      atomicAdd(&R.hist[nxt][(E + R.Nb) >> 1], 1u);
      lo = q;
    }
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
    if (R.model == 1) atomicAdd(&R.sumE2hi_next, hi);
  }
}

template <int TPB>
__global__ void __launch_bounds__(TPB) k_sweep_box(RunDev* __restrict__ runs, const Work* __restrict__ table,
                                                   int init) {
  extern __shared__ uint32_t smem[];
  const Work wk = table[blockIdx.x];
  RunDev& R = runs[wk.run];
  if (!init && R.skip) return;
  const int64_t Rn = init ? R.R : R.R_next;
  if ((int64_t)wk.first >= Rn) return;
  const int WR = R.Wr, W = R.W, S = R.bsites, model = R.model;
  const int plane = WR * S;
  int32_t* s_code = reinterpret_cast<int32_t*>(smem);
  int32_t* s_J = s_code + 14 * plane;
  int32_t* s_S = s_J + 12 * plane;
  __shared__ uint32_t s_thr[8];
  uint32_t* s_spin = reinterpret_cast<uint32_t*>(s_S + 2 * plane);
  const int tid = threadIdx.x;
  for (int i = tid; i < 14 * plane; i += TPB) s_code[i] = R.box_code[i];
  for (int i = tid; i < 12 * plane; i += TPB) s_J[i] = R.gJ[i];
  for (int i = tid; i < 2 * plane; i += TPB) s_S[i] = R.gS[i];
  if (tid < 8) s_thr[tid] = R.thr[tid];
  const int64_t slot = (int64_t)wk.first + tid;
  const bool live = slot < Rn;
  const int cur = R.cur, nxt = init ? 0 : cur ^ 1;
  uint32_t* col = s_spin + tid;
  const uint32_t valid = R.bvalid;
  if (live) {
    if (init) {
      for (int w4 = 0; w4 < W / 4; ++w4) {
        const u32x4 u = philox_seeded(R.seed, (uint32_t)w4, (uint32_t)slot, 0u, TAG_INIT);
        const uint32_t v[4] = {u.a, u.b, u.c, u.d};
        for (int i = 0; i < 4; ++i) {
          const int w = 4 * w4 + i;
          if (w < WR) col[w * TPB] = v[i] & valid;
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
  int E = 0;
  if (live) {
    if (!init) {
      const RoundKeys rk = make_round_keys(R.seed);
      const float beta_f = __double2float_rn(R.beta_next);
      const int theta = R.theta_next;
      const uint32_t T0 = (uint32_t)R.sweeps;
#pragma unroll 1
      for (int t = 0; t < theta; ++t) {
#pragma unroll 1
        for (uint32_t c = 0; c < 2; ++c)
          half_sweep_box<TPB>(col, s_code, s_J, s_S, WR, S, model, (uint32_t)slot, T0 + (uint32_t)t, c, rk,
                              s_thr, beta_f);
      }
    }
    E = energy_box<TPB>(col, s_code, s_J, WR, S, R.gC0);
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
  measure_box(R, nxt, slot, live, E);
}

// Dynamic shared memory of one block: the 28 table words per site pair
// (codes, couplings, sums) and the spin columns.
size_t box_smem_bytes(int WR, int S, int tpb) {
  return sizeof(int32_t) * (28 * (size_t)WR * S + (size_t)WR * tpb);
}

template <int TPB>
static cudaError_t launch_box_t(RunDev* runs, const Work* table, int nwork, int WR, int S, cudaStream_t st,
                                bool init) {
  const size_t sm = box_smem_bytes(WR, S, TPB);
  if (sm > BOX_SMEM_MAX) return nwork > 0 ? cudaErrorInvalidValue : cudaSuccess;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_box<TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (nwork <= 0) return cudaSuccess;
  k_sweep_box<TPB><<<nwork, TPB, sm, st>>>(runs, table, init ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_box(int tpb, RunDev* runs, const Work* table, int nwork, int WR, int S, cudaStream_t st,
                       bool init) {
  switch (tpb) {
    case 32: return launch_box_t<32>(runs, table, nwork, WR, S, st, init);
    case 64: return launch_box_t<64>(runs, table, nwork, WR, S, st, init);
    case 128: return launch_box_t<128>(runs, table, nwork, WR, S, st, init);
    case 256: return launch_box_t<256>(runs, table, nwork, WR, S, st, init);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pa
