// pa_divk.cuh -- x / k rounded to nearest (ties to even) for a double x >= 0
// and a small integer k, in integer arithmetic.
//
// The Poisson inverse-CDF walk (Sec. 2, resampling) divides by the step
// counter k at every step.  A double-precision division is a long chain of
// FP64 instructions, and on this GPU every FP64 instruction holds its SM
// sub-partition for about 64 cycles, so the walk spent most of its time in
// divisions.  The quotient of a 53-bit significand by k <= POISSON_KMAX is
// exact in 64-bit integer arithmetic, and rounding it to 53 bits by the IEEE
// rule gives the same double as any correctly rounded division:
//   x = M 2^e (M the 53-bit integer significand), n = M 2^11 in [2^63, 2^64);
//   q = floor(n / k) from the reciprocal floor(2^64 / k) (Granlund and
//   Montgomery, "Division by invariant integers using multiplication", PLDI
//   1994: the high half of n times the reciprocal is floor(n / k) or one
//   less, fixed by one remainder test);
//   keep the 53 leading bits of q; the dropped bits and the remainder decide
//   the rounding (above half: up; exactly half with remainder 0: to even).
// Zero, subnormal and non-finite x, and quotients that would be subnormal,
// are left to the division instruction.
// Included by exactly one translation unit (it owns the constant table).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pa_internal.h"

namespace pa {

// floor(2^64 / k) for 2 <= k <= POISSON_KMAX (entries 0 and 1 unused); the
// host fills it (set_division_table) before any launch.  Every lane of a
// warp in the walk reads the same k, so the constant cache broadcasts it.
__constant__ uint64_t c_recip_k[POISSON_KMAX + 1];

__device__ __forceinline__ double div_small_rn(double x, uint32_t k) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const int bexp = (int)(bits >> 52);  // biased exponent (sign bit clear for x >= 0)
  if (k == 1u && bexp < 0x7FF) return x;  // (the division would quiet a signalling NaN)
  if (bexp == 0 || bexp >= 0x7FF || k > (uint32_t)POISSON_KMAX) return __ddiv_rn(x, (double)k);
  const uint64_t n = ((bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
  uint64_t q = __umul64hi(n, c_recip_k[k]);
  uint64_t r = n - q * (uint64_t)k;
  if (r >= (uint64_t)k) {
    q += 1u;
    r -= (uint64_t)k;
  }
  // n / k >= 2^63 / 512 = 2^54 and < 2^63: 2 to 10 bits below the 53 kept
  const int sh = (63 - __clzll((long long)q)) - 52;
  int biased = bexp + sh - 11;  // exponent of the truncated quotient
  // a quotient below 2^-1022 rounds on the subnormal grid, not to 53 bits
  if (biased <= 0) return __ddiv_rn(x, (double)k);
  uint64_t mant = q >> sh;
  const uint64_t dropped = q & ((1ull << sh) - 1u);
  const uint64_t half = 1ull << (sh - 1);
  if (dropped > half || (dropped == half && (r != 0u || (mant & 1u)))) mant += 1u;
  if (mant == (1ull << 53)) {
    mant >>= 1;
    biased += 1;
  }
  return __longlong_as_double((long long)(((uint64_t)biased << 52) | (mant & 0x000FFFFFFFFFFFFFull)));
}

}  // namespace pa
