// pa_dexp.cuh -- deterministic double-precision exp for the step kernels.
// Included by exactly one translation unit (it owns the constant table).
#pragma once
#include "pa_device.cuh"

namespace pa {

// ---------------------------------------------------------------------------
// dexp_np: exp(x) for x <= 0, bit-reproducible.  Cody & Waite reduction
// x = k ln2 + r with a 40-bit head of ln2 (k*head exact for |k| < 2^13),
// degree-13 Taylor polynomial of exp(r) in Horner form with fused
// multiply-adds, |r| <= ln2/2 so the truncation error is below 2^-57, then
// scaling by 2^k (in two factors when 2^k would be subnormal).  The Taylor
// coefficients obey c_0 = 1, c_j = c_{j-1} / j with each quotient rounded to
// nearest; the host fills them (pa_set_exp_coefficients) before any launch.
//   head = floor(ln2 * 2^40) / 2^40, tail = ln2 - head (nearest),
//   1/ln2 rounded to nearest.
// ---------------------------------------------------------------------------
constexpr double DEXP_INV_LN2 = 0x1.71547652b82fep+0;
constexpr double DEXP_LN2_HEAD = 0x1.62e42fefa2000p-1;
constexpr double DEXP_LN2_TAIL = 0x1.9ef35793c7673p-41;
constexpr double DEXP_SHIFT = 0x1.8p52;
constexpr int DEXP_DEGREE = 13;

__constant__ double c_dexp_coef[DEXP_DEGREE + 1];

__device__ __forceinline__ double pow2_int(int k) {  // -1022 <= k <= 1023
  return __longlong_as_double((long long)(k + 1023) << 52);
}

__device__ __forceinline__ double dexp_np(double x) {
  if (x != x) return x;
  if (x > 0.0) return __longlong_as_double(0x7FF8000000000000LL);
  if (x < -746.0) return 0.0;
  const double t = __dmul_rn(x, DEXP_INV_LN2);
  const double kd = __dsub_rn(__dadd_rn(t, DEXP_SHIFT), DEXP_SHIFT);
  const double a = __dmul_rn(kd, DEXP_LN2_HEAD);
  const double b = __dsub_rn(x, a);
  const double c = __dmul_rn(kd, DEXP_LN2_TAIL);
  const double r = __dsub_rn(b, c);
  double p = c_dexp_coef[DEXP_DEGREE];
#pragma unroll
  for (int j = DEXP_DEGREE - 1; j >= 0; --j) p = __fma_rn(p, r, c_dexp_coef[j]);
  const int k = (int)kd;
  if (k >= -1022) return __dmul_rn(p, pow2_int(k));
  return __dmul_rn(__dmul_rn(p, pow2_int(k + 200)), pow2_int(-200));
}

// Uint32 Metropolis threshold for an energy rise dE > 0 at inverse temperature
// beta: floor(exp(-beta dE) 2^32), saturated at 2^32 - 1.
__device__ __forceinline__ uint32_t metropolis_threshold(double beta, int dE) {
  const double prob = dexp_np(-__dmul_rn(beta, (double)dE));
  const double scaled = __dmul_rn(prob, 4294967296.0);
  if (scaled >= 4294967296.0) return 0xFFFFFFFFu;
  return (uint32_t)scaled;
}

}  // namespace pa
