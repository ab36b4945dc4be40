// FP64 exp, expm1, log and log1p for the soil laws, table-driven after
// P. T. P. Tang, "Table-driven implementation of the exponential function in
// IEEE floating-point arithmetic" (ACM TOMS 15, 1989) and "Table-driven
// implementation of the logarithm function" (ACM TOMS 16, 1990).  On this GPU
// FP64 arithmetic issues at ~1/64 of the FP32 rate, and the laws of the FP64
// outer layer take six of these functions per cell, so they are written for
// few FP64 instructions: one table lookup and a short polynomial each.
//
//   exp:   x = (256 m + j) ln2/256 + r, j in [-128, 127], |r| <= ln2/512;
//          e^x = 2^m 2^(j/256) (1 + p(r)), p the Taylor polynomial of e^r - 1
//          to r^5 (truncation < 1e-20 absolute, < 7e-18 relative to r).
//   expm1: |x| < 1/128: the Taylor polynomial to x^7; m = 0: (2^(j/256) - 1)
//          + 2^(j/256) p(r) with 2^(j/256) - 1 from the table (no
//          cancellation); otherwise e^x - 1 (|x| > ln2/2: no significant
//          cancellation).
//   log:   |x - 1| < 1/128: the series of log1p below; otherwise
//          x = 2^e (1 + k/256) (1 + r), 0 <= r < 1/256; log x = e ln2 +
//          log(1 + k/256) + q(r), q the Taylor polynomial of log(1 + r) to r^7
//          (truncation < 7e-21 absolute); for k >= 128 the pair is taken as
//          (e + 1, (1 + k/256)/2), so that no large terms cancel below 1.
//   log1p: |s| < 1/128: the Taylor polynomial to s^10; s >= 1/128: log of
//          the rounded sum u = 1 + s plus the rounding remainder
//          (s - (u - 1)) / u.
// Results are within a few ulps of the correctly rounded values (tested
// against CUDA's functions).  Arguments outside the ranges the laws use
// (|x| > 700 for exp/expm1; non-normal or non-positive x for log; s <
// -1/128 for log1p) go to CUDA's functions.
#pragma once

#include "fp64_tables.h"

namespace rich {
namespace fx {

constexpr double SHIFT = 6755399441055744.0;   // 1.5 * 2^52: adding it rounds to an integer

// x = (256 m + j) ln2/256 + r
__device__ __forceinline__ void exp_reduce(double x, int& m, int& j, double& r) {
  const double t = fma(x, INV_LN2_256, SHIFT);
  const double nd = t - SHIFT;
  const int n = (int)(unsigned)__double2loint(t);
  j = ((n + 128) & 255) - 128;
  m = (n - j) >> 8;
  r = fma(-nd, LN2_256_HI, x);
  r = fma(-nd, LN2_256_LO, r);
}

// e^r - 1 for |r| <= ln2/512
__device__ __forceinline__ double expm1_poly(double r) {
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(r, p, 1.0 / 6.0);
  p = fma(r, p, 0.5);
  p = fma(r, p, 1.0);
  return r * p;
}

__device__ __forceinline__ double pow2i(int m) { return __hiloint2double((m + 1023) << 20, 0); }

__device__ __forceinline__ double exp(double x) {
  if (!(fabs(x) <= 700.0)) return ::exp(x);
  int m, j;
  double r;
  exp_reduce(x, m, j, r);
  const double p = expm1_poly(r);
  const double* T = kExp2[j + 128];
  return pow2i(m) * (T[0] + fma(T[0], p, T[1]));
}

__device__ __forceinline__ double expm1(double x) {
  const double ax = fabs(x);
  if (ax < 0.0078125) {
    // x + x^2/2 + ... + x^7/5040
    double p = fma(x, 1.0 / 5040.0, 1.0 / 720.0);
    p = fma(x, p, 1.0 / 120.0);
    p = fma(x, p, 1.0 / 24.0);
    p = fma(x, p, 1.0 / 6.0);
    p = fma(x, p, 0.5);
    p = fma(x, p, 1.0);
    return x * p;
  }
  if (!(ax <= 700.0)) return ::expm1(x);
  int m, j;
  double r;
  exp_reduce(x, m, j, r);
  const double p = expm1_poly(r);
  const double* T = kExp2[j + 128];
  if (m == 0) return T[2] + (T[3] + fma(T[0], p, T[1] * p));
  return fma(pow2i(m), T[0] + fma(T[0], p, T[1]), -1.0);
}

// log(1 + r) for 0 <= r < 1/256: r - r^2/2 + ... + r^7/7
__device__ __forceinline__ double log1p_poly7(double r) {
  double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
  q = fma(r, q, 1.0 / 5.0);
  q = fma(r, q, -1.0 / 4.0);
  q = fma(r, q, 1.0 / 3.0);
  q = fma(r, q, -0.5);
  return fma(r * r, q, r);
}

// log x for a positive normal x; *inv (nullable) receives an approximation
// of 1/x good to 1/256 relative
__device__ __forceinline__ double log_normal(double x, double* inv) {
  const int hi = __double2hiint(x);
  const int lo = __double2loint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023;
  const int k = (hi >> 12) & 255;                               // first 8 fraction bits
  const double M = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);   // in [1, 2)
  const double F = __hiloint2double(0x3ff00000 | (k << 12), 0);         // 1 + k/256
  const double* L = kLogF[k];
  const double rr = (M - F) * L[2];                             // (M - F)/F, M - F exact
  const double q = log1p_poly7(rr);
  if (inv) *inv = L[2] * pow2i(-e);
  const double ed = (double)(e + (k >> 7));                     // (k >= 128: the table holds log(F/2))
  return fma(ed, LN2_HI, L[0]) + (fma(ed, LN2_LO, L[1]) + q);
}

// log(1 + s) for |s| < 1/128: s - s^2/2 + s^3/3 - ... - s^10/10
__device__ __forceinline__ double log1p_series(double s) {
  double q = fma(s, -1.0 / 10.0, 1.0 / 9.0);
  q = fma(s, q, -1.0 / 8.0);
  q = fma(s, q, 1.0 / 7.0);
  q = fma(s, q, -1.0 / 6.0);
  q = fma(s, q, 1.0 / 5.0);
  q = fma(s, q, -1.0 / 4.0);
  q = fma(s, q, 1.0 / 3.0);
  q = fma(s, q, -0.5);
  return fma(s * s, q, s);
}

__device__ __forceinline__ double log(double x) {
  if (!(x >= 2.2250738585072014e-308 && x < 1.7976931348623157e308)) return ::log(x);
  const double s = x - 1.0;                  // exact near 1
  if (fabs(s) < 0.0078125) return log1p_series(s);
  return log_normal(x, nullptr);
}

// (the laws take log1p of non-negative arguments; s < -1/128 goes to CUDA's)
__device__ __forceinline__ double log1p(double s) {
  if (fabs(s) < 0.0078125) return log1p_series(s);
  if (s < 0.0) return ::log1p(s);
  const double u = 1.0 + s;
  if (!(u < 1.7976931348623157e308)) return ::log1p(s);
  const double c = s - (u - 1.0);            // what the rounded sum dropped
  double inv;
  const double l = log_normal(u, &inv);
  return l + c * inv;
}

}  // namespace fx
}  // namespace rich
