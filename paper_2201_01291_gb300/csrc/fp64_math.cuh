// FP64 exponential, logarithm and power of a positive base for the nodal closures of the FP64
// path (local-field mobility mu0 (|E| / E_ref)^p and Townsend alpha = A exp(-B/|E|)), with a
// few tens of FP64 operations each.  GB300 issues about one warp-wide FP64 instruction per 17
// cycles per SM, so general-purpose library routines, which handle every special case with full
// correct rounding, made these two closures most of the nodal kernel's time.  The arguments here
// are finite, the bases positive and normal.  exp and log are accurate to a few units in the
// last place; pow carries log's rounding times |p log x| (about 4e-16 (1 + |p log x|) relative),
// a few ulp for the mobility closure, whose |p log x| stays below 2 (tested against the CUDA
// math library on the device).
//
//   exp: Cody-Waite argument reduction x = n ln2 + r, |r| <= ln2 / 2, with ln2 split in a head
//        of 32 significant bits (n ln2_hi exact for |n| < 2^21) and a tail; e^r by its Taylor
//        polynomial of degree 12 (truncation below 2e-16 relative at |r| = ln2 / 2), Horner form;
//        2^n put in the exponent field (results below the smallest normal flush to zero).
//   log: x = m 2^e with m in [sqrt(1/2), sqrt(2)); log m = 2 atanh(s), s = (m - 1) / (m + 1),
//        |s| <= 0.1716, by the odd series 2 (s + s^3/3 + ... + s^21/21) (truncation below 1e-18);
//        1 / (m + 1) by two Newton-Raphson steps y <- y (2 - d y) from the FP32 reciprocal.
//   pow: x^p = exp(p log x), x > 0.
#pragma once

namespace avip {

__device__ __forceinline__ double exp_fp64(double x) {
  constexpr double kLog2e = 1.4426950408889634;
  constexpr double kLn2Hi = 0.6931471806019545;      // ln 2 rounded to 32 significant bits
  constexpr double kLn2Lo = -4.2009150726810846e-11;  // ln 2 - kLn2Hi
  if (x > 709.0) return __longlong_as_double(0x7ff0000000000000LL);  // overflow: +inf
  if (x < -708.0) return 0.0;                                          // below the normal range
  const double n = rint(x * kLog2e);
  double r = fma(-n, kLn2Hi, x);
  r = fma(-n, kLn2Lo, r);
  // e^r = sum_k r^k / k!, k = 0 .. 12 (coefficients 1/k!)
  double p = 1.0 / 479001600.0;
  p = fma(p, r, 1.0 / 39916800.0);
  p = fma(p, r, 1.0 / 3628800.0);
  p = fma(p, r, 1.0 / 362880.0);
  p = fma(p, r, 1.0 / 40320.0);
  p = fma(p, r, 1.0 / 5040.0);
  p = fma(p, r, 1.0 / 720.0);
  p = fma(p, r, 1.0 / 120.0);
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = fma(p, r, 1.0);
  const long long bits = (long long)((int)n + 1023) << 52;  // 2^n, n in [-1022, 1023]
  return p * __longlong_as_double(bits);
}

__device__ __forceinline__ double log_fp64(double x) {
  constexpr double kLn2Hi = 0.6931471806019545;
  constexpr double kLn2Lo = -4.2009150726810846e-11;
  constexpr double kSqrt2 = 1.4142135623730951;
  long long bits = __double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7ff) - 1023;
  double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);  // [1, 2)
  if (m > kSqrt2) {
    m *= 0.5;
    e += 1;
  }
  const double d = m + 1.0;
  double y = (double)__frcp_rn((float)d);
  y = y * fma(-d, y, 2.0);
  y = y * fma(-d, y, 2.0);
  const double s = (m - 1.0) * y;
  const double s2 = s * s;
  // atanh(s) / s = sum_k s^2k / (2k + 1), k = 0 .. 10
  double t = 1.0 / 21.0;
  t = fma(t, s2, 1.0 / 19.0);
  t = fma(t, s2, 1.0 / 17.0);
  t = fma(t, s2, 1.0 / 15.0);
  t = fma(t, s2, 1.0 / 13.0);
  t = fma(t, s2, 1.0 / 11.0);
  t = fma(t, s2, 1.0 / 9.0);
  t = fma(t, s2, 1.0 / 7.0);
  t = fma(t, s2, 1.0 / 5.0);
  t = fma(t, s2, 1.0 / 3.0);
  t = fma(t, s2, 1.0);
  const double lm = 2.0 * s * t;
  const double ed = (double)e;
  return fma(ed, kLn2Hi, fma(ed, kLn2Lo, lm));
}

__device__ __forceinline__ double pow_pos_fp64(double x, double p) { return exp_fp64(p * log_fp64(x)); }

// 1 / d for a nonzero d: the hardware's approximate reciprocal refined by two Newton-Raphson
// steps y <- y + y (1 - d y) (each squares the relative error: about 2^-20 -> 2^-40 -> the FP64
// rounding), within a few ulp of the rounded quotient, for 5 FP64 instructions against about
// twice that for an IEEE division.  A subnormal d (exponent field zero; the approximation
// flushes it) takes the division.
__device__ __forceinline__ double recip_nr(double d) {
  if ((__double2hiint(d) & 0x7ff00000) == 0) return 1.0 / d;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  double e = fma(-d, y, 1.0);
  y = fma(y, e, y);
  e = fma(-d, y, 1.0);
  return fma(y, e, y);
}

}  // namespace avip
