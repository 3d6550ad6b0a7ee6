// Table-driven FP64 elementary functions for the model evaluation.
//
// On GB300 every FP64 instruction costs about 64 FP32 instruction slots, and the evaluation is
// bound by the FP64 pipe, so the three transcendental calls of a device (exp and log1p in the
// effective overdrive, expm1 in each junction) are worth specialising. The methods are P. T. P.
// Tang's table-driven algorithms:
//   exp   — "Table-driven implementation of the exponential function in IEEE floating-point
//           arithmetic", ACM TOMS 15(2), 1989: x = (256 m + j) ln2/256 + r with |r| <= ln2/512
//           (Cody–Waite reduction with a two-part ln2/256), exp(x) = 2^m 2^(j/256) e^r, e^r - 1
//           by its Taylor polynomial (256 entries rather than Tang's 32: one degree less);
//   expm1 — "Table-driven implementation of the expm1 function ...", ACM TOMS 18(2), 1992: a
//           Taylor polynomial for small |x|, otherwise the exp reduction with 2^(j/256) held as a
//           double-double so that (2^m T - 1) is formed without losing the leading bits;
//   log1p — "Table-driven implementation of the logarithm function ...", ACM TOMS 16(4), 1990,
//           specialised to 1 + e with e in [0, 1]: y = 1 + e, F = 1 + j/256 nearest to y,
//           u = (y - F)/F, log y = log F + log1p(u) by its Taylor polynomial, plus the rounding
//           error of 1 + e carried as c / y. One path for the whole interval (j = 0, F = 1
//           covers small e, where the polynomial's truncation stays below 2^-54 relative to
//           log y): a branch for small e would be taken by some lanes of most warps.
// Reciprocal and reciprocal square root start from the FP32 special-function unit and finish
// with one third-order correction from the series of 1/(1 - e) and (1 - e)^(-1/2).
// Polynomial coefficients are Taylor coefficients; tables come from gen_tables.py. Accuracy
// (checked against CUDA's functions by the GPU tests through eec_math_check) is within a few
// units in the last place over the domains used here (1 ulp for the reciprocal, 2 for rsqrt).
#pragma once

#include <cuda_runtime.h>

#include "eec_tables.h"

namespace eec {

// Comparisons on the bit pattern. For every non-NaN argument each one decides exactly as the
// floating-point comparison in its name, but runs on the integer pipe: a double compare would
// occupy the FP64 pipe, which bounds the evaluation.
constexpr long long kBits40 = 0x4044000000000000LL;            // 40.0
constexpr long long kBits709 = 0x4086280000000000LL;           // 709.0
constexpr unsigned long long kBits707 = 0x4086180000000000ull;  // 707.0
constexpr unsigned long long kBitsM38 = 0xC043000000000000ull;  // -38.0
constexpr unsigned long long kBits2m6 = 0x3F90000000000000ull;  // 2^-6
constexpr long long kBits2m7 = 0x3F80000000000000LL;           // 2^-7

__device__ __forceinline__ unsigned long long fm_ubits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}
// x >= 0.0 (true at -0.0): the sign bit is clear, or x is -0.0
__device__ __forceinline__ bool fm_ge0(double x) { return fm_ubits(x) <= 0x8000000000000000ull; }
// x < c, x <= c for a constant c > 0 (negative x, -0.0 included, are negative as integers)
__device__ __forceinline__ bool fm_lt_pos(double x, long long cbits) {
  return __double_as_longlong(x) < cbits;
}
__device__ __forceinline__ bool fm_le_pos(double x, long long cbits) {
  return __double_as_longlong(x) <= cbits;
}
// x < c for a constant c < 0 (below c means a larger magnitude with the sign bit set)
__device__ __forceinline__ bool fm_lt_neg(double x, unsigned long long cbits) {
  return fm_ubits(x) > cbits;
}
// |x| < c for a constant c > 0
__device__ __forceinline__ bool fm_abs_lt(double x, unsigned long long cbits) {
  return (fm_ubits(x) & 0x7fffffffffffffffull) < cbits;
}

// x * 2^k by adding k to the exponent field (integer pipe). Exact whenever x and the result are
// normal; x with a zero exponent field (+-0, subnormals below 2.3e-308) or an all-ones one
// (inf, NaN) is returned unchanged.
__device__ __forceinline__ double fm_pow2(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  return (e == 0 || e == 0x7ff) ? x : __longlong_as_double(b + ((long long)k << 52));
}

// Seeds from the FP32 special-function unit. The double x is narrowed on the integer pipe from its
// high word (sign, exponent rebiased by 1023 - 127, top 20 mantissa bits; relative error below
// 2^-20, valid for 2^-126 <= |x| < 2^128), the approximation widened back the same way.
__device__ __forceinline__ float fm_narrow(double x) {
  const int hi = __double2hiint(x);
  return __int_as_float((((hi & 0x7fffffff) - 0x38000000) << 3) | (hi & 0x80000000));
}
__device__ __forceinline__ double fm_widen(float f) {
  const int b = __float_as_int(f);
  return __hiloint2double((((b & 0x7fffffff) >> 3) + 0x38000000) | (b & 0x80000000), 0);
}

// 1/x by one third-order Newton step from the seed y0 (relative error e0 below 2^-19):
// with e = 1 - x y0, 1/x = y0 / (1 - e) = y0 (1 + e + e^2 + ...), so y0 + y0 (e + e^2) leaves
// a relative error of e0^3 < 2^-57 plus the rounding of the last two operations.
// For normal |x| in [2^-126, 2^128) (the model's denominators are far inside).
__device__ __forceinline__ double fm_rcp(double x) {
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(fm_narrow(x)));
  const double y0 = fm_widen(yf);
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}

// 1/sqrt(x) by one third-order step: with e = 1 - x y0^2, x^(-1/2) = y0 (1 - e)^(-1/2)
// = y0 (1 + e/2 + 3 e^2/8 + ...); the truncation leaves 5 e0^3 / 16.
__device__ __forceinline__ double fm_rsqrt(double x) {
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(fm_narrow(x)));
  const double y0 = fm_widen(yf);
  const double e = fma(-x * y0, y0, 1.0);
  return fma(y0, e * fma(e, 0.375, 0.5), y0);
}

// y * 2^m by adding m to the exponent field (y and the result must be normal, y != 0).
__device__ __forceinline__ double fm_scale2(double y, int m) {
  return __hiloint2double(__double2hiint(y) + (m << 20), __double2loint(y));
}

// Argument reduction shared by exp and expm1: x = (256 m + j) ln2/256 + r.
static_assert(kExpN == 256, "fm_reduce splits n into 8 table bits and the exponent");
__device__ __forceinline__ double fm_reduce(double x, int& j, int& m) {
  const double s = fma(x, kInvLn2xN, 0x1.8p52);   // 1.5 * 2^52 shifter: rounds x*256/ln2
  const int n = __double2loint(s);
  const double nf = s - 0x1.8p52;
  j = n & (kExpN - 1);
  m = n >> 8;
  return fma(-nf, kLn2oNLo, fma(-nf, kLn2oNHi, x));
}

// e^r - 1 for |r| <= ln2/512: Taylor polynomial through r^4 (truncation 3.8e-17, below 0.2 ulp
// of e^r; enough for exp, whose result is near 1).
__device__ __forceinline__ double fm_em1_small(double r) {
  const double q = fma(r, fma(r, fma(r, 1.0 / 24.0, 1.0 / 6.0), 0.5), 1.0);
  return r * q;
}

// The same through r^5 (truncation 9e-21): expm1 results can be as small as 2^-6, so the
// polynomial error must stay below their ulp.
__device__ __forceinline__ double fm_em1_small5(double r) {
  const double q = fma(r, fma(r, fma(r, fma(r, 1.0 / 120.0, 1.0 / 24.0), 1.0 / 6.0), 0.5), 1.0);
  return r * q;
}

__device__ __forceinline__ double fm_exp(double x) {
  if (!fm_abs_lt(x, kBits707)) return ::exp(x);   // near the subnormal / overflow range, NaN
  int j, m;
  const double r = fm_reduce(x, j, m);
  const double p = fm_em1_small(r);
  const double th = __ldg(kExp2Hi + j);
  const double y = fma(th, p, __ldg(kExp2Lo + j)) + th;   // 2^(j/256) e^r in [0.997, 2)
  return fm_scale2(y, m);
}

__device__ __forceinline__ double fm_expm1(double x) {
  if (fm_abs_lt(x, kBits2m6)) {
    // x + x^2/2 + ... + x^7/5040 (truncation below 2^-59 relative)
    const double q = fma(x, fma(x, fma(x, fma(x, fma(x, 1.0 / 5040.0, 1.0 / 720.0), 1.0 / 120.0),
                                       1.0 / 24.0), 1.0 / 6.0), 0.5);
    return fma(x * x, q, x);
  }
  if (fm_lt_neg(x, kBitsM38)) return -1.0;   // e^x < 2^-54: -1 + e^x rounds to -1
  if (!fm_lt_pos(x, kBits709)) return ::expm1(x);
  int j, m;
  const double r = fm_reduce(x, j, m);
  const double p = fm_em1_small5(r);
  const double T = fm_scale2(__ldg(kExp2Hi + j), m);
  const double tl = __ldg(kExp2Lo + j);
  const double Tl = (__double2hiint(tl) == 0 && __double2loint(tl) == 0) ? 0.0 : fm_scale2(tl, m);
  return (T - 1.0) + fma(T, p, Tl);
}

// log(1 + e) for e in [0, 1]; inv_y must be 1 / (1 + e) rounded (the caller needs it anyway).
__device__ __forceinline__ double fm_log1p01(double e, double inv_y) {
  const double y = 1.0 + e;                        // [1, 2]
  const double c = e - (y - 1.0);                  // rounding error of y, exact
  const double s = fma(y, (double)kLogN, 0x1.8p52);   // round(256 y) in [256, 512]
  const int jj = __double2loint(s) - kLogN;        // F = 1 + jj/256, jj in [0, 256]
  const double u = (y - __ldg(kF + jj)) * __ldg(kInvF + jj);   // |u| <= 2^-9; y - F exact
  const double q = fma(u, fma(u, fma(u, fma(u, -1.0 / 6.0, 0.2), -0.25), 1.0 / 3.0), -0.5);
  const double pu = fma(u * u, q, u);              // log1p(u), truncation below 2^-54 relative
  return __ldg(kLogFHi + jj) + fma(c, inv_y, __ldg(kLogFLo + jj) + pu);
}

}  // namespace eec
