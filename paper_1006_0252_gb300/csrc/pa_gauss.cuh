// pa_gauss.cuh -- population annealing with Gaussian couplings (the model of
// the paper's Sec. 4), fixed point: physical J = J_q * 2^-15, so energies and
// energy changes are exact integers.
//
// Metropolis rise dE_q > 0 at beta: accept iff float(u >> 8) < fexp(x) * 2^24,
// x = -(float(beta) * float(dE_q)) * 2^-15, every operation explicitly
// rounded; fexp is the deterministic single-precision exp below.
#pragma once
#include "pa_device.cuh"

namespace pa {

constexpr float GAUSS_INV_SCALE = 0x1.0p-15f;
constexpr double GAUSS_INV_SCALE_D = 0x1.0p-15;

// fexp: exp(x) for x <= 0 in single precision, bit-reproducible.  Cody & Waite
// reduction with a 16-bit head of ln2 (k * head exact for |k| <= 151), Taylor
// polynomial of degree 7 in Horner form with fused multiply-adds, scaling by
// 2^k in two factors below the normal range; coefficients c_0 = 1,
// c_j = c_{j-1} / j rounded to single precision (computed here at compile time:
// single-precision division of small exact integers is correctly rounded).
//   head = floor(ln2 * 2^16) / 2^16, tail = ln2 - head (nearest float),
//   1/ln2 to nearest float.
constexpr float FEXP_INV_LN2 = 0x1.715476p+0f;
constexpr float FEXP_LN2_HEAD = 0x1.62e4p-1f;
constexpr float FEXP_LN2_TAIL = 0x1.7f7d1cp-20f;
constexpr float FEXP_SHIFT = 0x1.8p23f;

__device__ __forceinline__ float pow2f_int(int k) {  // -126 <= k <= 127
  return __int_as_float((k + 127) << 23);
}

__device__ __forceinline__ float fexp_np(float x) {
  if (x < -104.0f) return 0.0f;
  const float t = __fmul_rn(x, FEXP_INV_LN2);
  const float kf = __fsub_rn(__fadd_rn(t, FEXP_SHIFT), FEXP_SHIFT);
  const float a = __fmul_rn(kf, FEXP_LN2_HEAD);
  const float b = __fsub_rn(x, a);
  const float c = __fmul_rn(kf, FEXP_LN2_TAIL);
  const float r = __fsub_rn(b, c);
  // c_j = c_{j-1} / j in single precision: 1, 1, 1/2, 1/6, 1/24, 1/120, 1/720, 1/5040
  constexpr float c2 = 1.0f / 2.0f, c3 = c2 / 3.0f, c4 = c3 / 4.0f, c5 = c4 / 5.0f, c6 = c5 / 6.0f,
                  c7 = c6 / 7.0f;
  float p = c7;
  p = __fmaf_rn(p, r, c6);
  p = __fmaf_rn(p, r, c5);
  p = __fmaf_rn(p, r, c4);
  p = __fmaf_rn(p, r, c3);
  p = __fmaf_rn(p, r, c2);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  const int k = (int)kf;
  if (k >= -126) return __fmul_rn(p, pow2f_int(k));
  return __fmul_rn(__fmul_rn(p, pow2f_int(k + 64)), pow2f_int(-64));
}

// Metropolis decision for a site with integer energy change dE at beta (float)
__device__ __forceinline__ bool gauss_accept(int dE, float beta_f, uint32_t u) {
  if (dE <= 0) return true;
  const float x = -__fmul_rn(__fmul_rn(beta_f, __int2float_rn(dE)), GAUSS_INV_SCALE);
  const float lim = __fmul_rn(fexp_np(x), 16777216.0f);
  return __uint2float_rn(u >> 8) < lim;
}

// The same decision as an integer threshold: u >> 8 is an integer below
// 2^24, exactly representable, so float(u >> 8) < lim <=> (u >> 8) < ceil(lim)
// for a float lim in [0, 2^24]; gauss_accept(dE, beta_f, u) is therefore
// (u >> 8) < gauss_threshold(dE, beta_f), with 2^24 (always) for dE <= 0.
__device__ __forceinline__ uint32_t gauss_threshold(int dE, float beta_f) {
  if (dE <= 0) return 1u << 24;
  const float x = -__fmul_rn(__fmul_rn(beta_f, __int2float_rn(dE)), GAUSS_INV_SCALE);
  return __float2uint_ru(__fmul_rn(fexp_np(x), 16777216.0f));
}

__device__ __forceinline__ float ex2_approx_ftz(float y) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}

// The same decision as gauss_accept, settled first against a hardware
// estimate t of fexp(x) 2^24: y = -(beta (log2(e) 2^-15)) dE carries at most
// 3 roundings of 2^-24 relative (plus the constant's 2^-25), so for the
// |y| <= 150 where the estimate is not flushed to zero, 2^y is within
// 150 * 3.5 * 2^-24 * ln 2 < 2.2e-5 relative of exp(x); ex2.approx and
// fexp's 2 ulp add < 1e-6.  A window of 2^-12 (2.4e-4) around t therefore
// holds every u24 whose exact decision could differ; only inside it, and for
// u24 = 0 against a flushed estimate, is fexp evaluated.
constexpr float GAUSS_LOG2E_SCALED = 0x1.715476p+0f * 0x1.0p-15f;  // log2(e) 2^-15
// 2^24 (1 -+ 2^-12), exact in binary32: the window around the estimate.
constexpr float GAUSS_WIN_LO = 16773120.0f;
constexpr float GAUSS_WIN_HI = 16781312.0f;

// acc += J where bit `MASK` of x is set: a one-instruction bit test on the
// integer ALU and a predicated multiply-add (J * one + acc, one == 1 at run
// time) on the multiply-add pipe.
template <uint32_t MASK>
__device__ __forceinline__ void add_if_set(int32_t& acc, uint32_t x, int32_t J, uint32_t one) {
  asm("{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t"
      "and.b32 t, %1, %2;\n\t"
      "setp.ne.u32 p, t, 0;\n\t"
      "@p mad.lo.s32 %0, %3, %4, %0;\n\t}"
      : "+r"(acc)
      : "r"(x), "n"(MASK), "r"(J), "r"(one));
}

// The same with the bit mask in a register (ranks from an unrolled loop).
__device__ __forceinline__ void add_if_set(int32_t& acc, uint32_t x, uint32_t mask, int32_t J, uint32_t one) {
  asm("{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t"
      "and.b32 t, %1, %2;\n\t"
      "setp.ne.u32 p, t, 0;\n\t"
      "@p mad.lo.s32 %0, %3, %4, %0;\n\t}"
      : "+r"(acc)
      : "r"(x), "r"(mask), "r"(J), "r"(one));
}

// Branch-free form of gauss_accept_fast for one site, bc = RN32(beta_f
// log2(e) 2^-15): sets bit `bit` of *flip where the decision is settled as an
// acceptance and of *amb where u24 falls inside the window (decide those with
// gauss_accept).  A rise dE > 0 outside the window with no flip bit is a
// rejection.
__device__ __forceinline__ void gauss_site(int dE, float bc, uint32_t u, uint32_t bit, uint32_t one, uint32_t* flip,
                                           uint32_t* amb) {
  const float t = ex2_approx_ftz(-__fmul_rn(bc, __int2float_rn(dE)));
  const float u24 = __uint2float_rn(u >> 8);
  const float lo = __fmul_rn(t, GAUSS_WIN_LO), hi = __fmul_rn(t, GAUSS_WIN_HI);
  // the decision as predicates; the two bit sets as predicated multiply-adds
  // (bit * one + mask; the ranks' bits are distinct) on the multiply-add pipe
  asm("{\n\t.reg .pred r, b, a, nr, nb, na, pf, pa;\n\t"
      "setp.gt.s32 r, %2, 0;\n\t"
      "setp.lt.f32 b, %3, %4;\n\t"
      "setp.gt.f32 a, %3, %5;\n\t"
      "not.pred nr, r;\n\t"
      "not.pred nb, b;\n\t"
      "not.pred na, a;\n\t"
      "or.pred pf, nr, b;\n\t"
      "and.pred pa, r, nb;\n\t"
      "and.pred pa, pa, na;\n\t"
      "@pf mad.lo.u32 %0, %6, %7, %0;\n\t"
      "@pa mad.lo.u32 %1, %6, %7, %1;\n\t}"
      : "+r"(*flip), "+r"(*amb)
      : "r"(dE), "f"(u24), "f"(lo), "f"(hi), "r"(bit), "r"(one));
}
__device__ __forceinline__ bool gauss_accept_fast(int dE, float beta_f, uint32_t u) {
  if (dE <= 0) return true;
  const float t = __fmul_rn(ex2_approx_ftz(-__fmul_rn(__fmul_rn(beta_f, GAUSS_LOG2E_SCALED), __int2float_rn(dE))),
                            16777216.0f);
  const float u24 = __uint2float_rn(u >> 8);
  if (u24 < __fmul_rn(t, 1.0f - 0x1.0p-12f)) return true;
  if (u24 > __fmul_rn(t, 1.0f + 0x1.0p-12f)) return false;
  return gauss_accept(dE, beta_f, u);
}

}  // namespace pa
