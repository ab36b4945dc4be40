// Float-float ("double-float") evaluation of the constitutive laws.
//
// GB300's FP64 pipe issues about 1/64 of the FP32 rate, so the FP64 special
// functions of theta(psi) and K(psi) dominate every FP64 kernel.  Here a value
// is an unevaluated sum hi + lo of two floats (~48 significant bits), built
// from the error-free transformations two-sum and two-product (Dekker 1971,
// Knuth): the results agree with FP64 evaluation to ~1e-14 relative, far
// inside the 1e-8 stop test and the 1e-12 stage tolerance, at a small
// fraction of the FP64 cost.
//
//   exp:  table-driven reduction by ln2/32 (Tang's method), a short Taylor
//         series for the remainder, then the exact scaling by 2^m;
//   expm1 of a small argument: the remainder scaled by 1/16, Taylor to
//         degree 7, four doublings y <- y (y + 2);
//   log:  one Newton step on exp from the single-precision logf:
//         log x = y0 + log1p(x e^{-y0} - 1), the log1p of a ~1e-7 argument
//         taken to second order;
//   log1p: the same Newton step on expm1 from log1pf.
#pragma once

#include "device.cuh"

namespace rich {

struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd mk(float h, float l = 0.0f) {
  dd r;
  r.hi = h;
  r.lo = l;
  return r;
}

// s + e = a + b exactly
__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return mk(s, e);
}

// s + e = a + b exactly, for |a| >= |b|
__device__ __forceinline__ dd quick_two_sum(float a, float b) {
  const float s = a + b;
  return mk(s, b - (s - a));
}

// p + e = a b exactly
__device__ __forceinline__ dd two_prod(float a, float b) {
  const float p = a * b;
  return mk(p, fmaf(a, b, -p));
}

__device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  const dd t = two_sum(x.lo, y.lo);
  s = quick_two_sum(s.hi, s.lo + t.hi);
  return quick_two_sum(s.hi, s.lo + t.lo);
}

__device__ __forceinline__ dd dd_neg(dd x) { return mk(-x.hi, -x.lo); }

__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  const dd p = two_prod(x.hi, y.hi);
  return quick_two_sum(p.hi, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo)));
}

__device__ __forceinline__ dd dd_mul_f(dd x, float f) {
  const dd p = two_prod(x.hi, f);
  return quick_two_sum(p.hi, fmaf(x.lo, f, p.lo));
}

__device__ __forceinline__ dd dd_from(double x) {
  const float h = __double2float_rn(x);
  return mk(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double dd_to(dd x) { return (double)x.hi + (double)x.lo; }

// ln 2 = C1 + C2 + C3 (C1 with 12 trailing zero bits: k C1 exact for |k| < 4096)
#define RICH_LN2_C1 0x1.62e000p-1f
#define RICH_LN2_C2 0x1.0bfbe8p-15f
#define RICH_LN2_C3 0x1.cf79acp-40f
#define RICH_INV_LN2 0x1.715476p+0f
#define RICH_INV6_HI 0x1.555556p-3f
#define RICH_INV6_LO -0x1.555556p-28f
#define RICH_INV24_HI 0x1.555556p-5f
#define RICH_INV24_LO -0x1.555556p-30f

// expm1(r) for |r| <= ln2/32: Taylor series, degree 7
__device__ __forceinline__ dd dd_expm1_reduced(dd r) {
  const float rf = r.hi;
  const float T = fmaf(rf, fmaf(rf, 1.0f / 5040.0f, 1.0f / 720.0f), 1.0f / 120.0f);   // r^5 coefficient tail
  dd c = dd_add(mk(RICH_INV24_HI, RICH_INV24_LO), dd_mul_f(r, T));
  c = dd_add(mk(RICH_INV6_HI, RICH_INV6_LO), dd_mul(r, c));
  c = dd_add(mk(0.5f), dd_mul(r, c));
  c = dd_add(mk(1.0f), dd_mul(r, c));
  return dd_mul(r, c);
}

// expm1 of x / 2^k-reduced argument, doubled back four times
__device__ __forceinline__ dd dd_expm1_core(dd r) {
  dd y = dd_expm1_reduced(mk(r.hi * 0.0625f, r.lo * 0.0625f));
  for (int k = 0; k < 4; ++k) y = dd_mul(y, dd_add(y, mk(2.0f)));    // e^{2s} - 1 = y (y + 2)
  return y;
}

// 2^(j/32), j = 0..31, as float pairs (hi + lo within 1.5e-15 relative)
static __device__ const float2 kExp2Frac[32] = {
    {0x1.000000p+0f, 0x0.0p+0f},          {0x1.059b0ep+0f, -0x1.9d4f52p-25f},
    {0x1.0b5586p+0f, 0x1.9f3122p-25f},    {0x1.11301ep+0f, -0x1.fdb496p-25f},
    {0x1.172b84p+0f, -0x1.c15742p-27f},   {0x1.1d4874p+0f, -0x1.d2e8cap-25f},
    {0x1.2387a6p+0f, 0x1.ceac48p-25f},    {0x1.29e9e0p+0f, -0x1.5c0424p-25f},
    {0x1.306fe0p+0f, 0x1.4636e2p-25f},    {0x1.371a74p+0f, -0x1.18aac6p-25f},
    {0x1.3dea64p+0f, 0x1.824684p-25f},    {0x1.44e086p+0f, 0x1.8624b4p-30f},
    {0x1.4bfdaep+0f, -0x1.593abcp-25f},   {0x1.5342b6p+0f, -0x1.2c5610p-25f},
    {0x1.5ab07ep+0f, -0x1.5bd5ecp-27f},   {0x1.6247ecp+0f, -0x1.f8b550p-25f},
    {0x1.6a09e6p+0f, 0x1.9fcef4p-26f},    {0x1.71f75ep+0f, 0x1.1d8beep-25f},
    {0x1.7a1148p+0f, -0x1.829fd0p-25f},   {0x1.82589ap+0f, -0x1.accc7cp-26f},
    {0x1.8ace54p+0f, 0x1.15506ep-27f},    {0x1.93737cp+0f, -0x1.e64744p-25f},
    {0x1.9c4918p+0f, 0x1.51f848p-27f},    {0x1.a5503cp+0f, -0x1.b83b54p-25f},
    {0x1.ae89fap+0f, -0x1.a94b14p-26f},   {0x1.b7f770p+0f, -0x1.a09438p-25f},
    {0x1.c199bep+0f, -0x1.3d56b2p-27f},   {0x1.cb720ep+0f, -0x1.8837ccp-27f},
    {0x1.d5818ep+0f, -0x1.822dbcp-27f},   {0x1.dfc974p+0f, -0x1.908c94p-25f},
    {0x1.ea4afap+0f, 0x1.52486cp-27f},    {0x1.f50766p+0f, -0x1.246eb0p-26f}};

// e^x for |x| <= ~70 (the scale and the low word stay normal floats):
// table-driven reduction (Tang's method) x = (32 m + j) ln2/32 + r,
// |r| <= ln2/64, with ln2/32 in three floats (the first with 12 significant
// bits, so k times it is exact for |k| < 4096); e^r - 1 by its Taylor series
// (terms to r^3 in float-float, r^4 .. r^6 in float); e^x = 2^m 2^(j/32)(1 + p).
__device__ __forceinline__ dd dd_exp(dd x) {
  const float kf = rintf(x.hi * (32.0f * RICH_INV_LN2));
  const int k = (int)kf;
  dd r = dd_add(x, mk(-kf * (RICH_LN2_C1 * 0.03125f)));
  r = dd_add(r, dd_neg(two_prod(kf, RICH_LN2_C2 * 0.03125f)));
  r = dd_add(r, mk(-kf * (RICH_LN2_C3 * 0.03125f)));
  const float rf = r.hi;
  const float q = rf * rf * fmaf(rf, fmaf(rf, 1.0f / 720.0f, 1.0f / 120.0f), 1.0f / 24.0f);
  dd b = dd_add(mk(0.5f), dd_mul(r, mk(RICH_INV6_HI, RICH_INV6_LO)));
  b = dd_add(b, mk(q));
  const dd p = dd_add(r, dd_mul(dd_mul(r, r), b));       // e^r - 1
  const float2 t = kExp2Frac[k & 31];
  const dd T = mk(t.x, t.y);
  const dd e = dd_add(T, dd_mul(T, p));
  const float s = __int_as_float((127 + (k >> 5)) << 23);   // 2^m, m = floor(k/32)
  return mk(e.hi * s, e.lo * s);
}

// e^x - 1, accurate relative to itself also for small |x|
__device__ __forceinline__ dd dd_expm1(dd x) {
  if (fabsf(x.hi) < 0.34657359f) return dd_expm1_core(x);
  return dd_add(dd_exp(x), mk(-1.0f));
}

// log x for x > 0
__device__ __forceinline__ dd dd_log(dd x) {
  const float y0 = logf(x.hi);
  const dd t = dd_mul(x, dd_exp(mk(-y0)));
  const dd d = dd_add(t, mk(-1.0f));                    // |d| ~ 1e-7
  const dd corr = dd_add(d, mk(-0.5f * d.hi * d.hi));
  return dd_add(mk(y0), corr);
}

// log(1 + t) for t > -1, accurate relative to itself also for small |t|:
// one Newton step on expm1 from the single-precision log1pf,
//   log1p t = y0 + log1p((t - expm1 y0) / (1 + expm1 y0)),
// the correction d ~ 1e-7 relative taken to second order (its float factor
// 1/(1 + expm1 y0) costs ~1e-7 of d, i.e. ~1e-14 of the result).
__device__ __forceinline__ dd dd_log1p(dd t) {
  const float y0 = log1pf(t.hi);
  const dd E = dd_expm1(mk(y0));
  const dd d = dd_mul_f(dd_add(t, dd_neg(E)), 1.0f / (1.0f + E.hi));
  return dd_add(mk(y0), dd_add(d, mk(-0.5f * d.hi * d.hi)));
}

// 1 / t (one Newton step from the float reciprocal)
__device__ __forceinline__ dd dd_recip(dd t) {
  const float r0 = 1.0f / t.hi;
  const dd e = dd_add(mk(1.0f), dd_neg(dd_mul_f(t, r0)));
  return dd_add(mk(r0), dd_mul_f(e, r0));
}

// ---------------------------------------------------------------------------
// FP64 <-> float-float.  FP64 arithmetic and FP32/FP64 conversions both issue
// at ~1/64 of the FP32 rate here, so a double is split with integer
// operations: hi = x truncated to 24 significant bits, lo = the next 23 bits
// (x - hi - lo < 2^-46 |x|).  |x| outside [2^-103, 2^128) (zero included)
// takes the conversion instead.
// ---------------------------------------------------------------------------
__device__ __forceinline__ dd dd_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu) - 1023 + 127;     // FP32 biased exponent of hi
  if (e >= 24 && e <= 254) {
    const unsigned fhi = ((hw & 0xfffffu) << 3) | (lw >> 29);  // fraction bits 51..29
    const unsigned flo = (lw >> 6) & 0x7fffffu;                // fraction bits 28..6
    const unsigned elo = (unsigned)(e - 23) << 23;
    const float one = __uint_as_float(sign | elo);
    return mk(__uint_as_float(sign | ((unsigned)e << 23) | fhi), __uint_as_float(sign | elo | flo) - one);
  }
  if ((b << 1) == 0ull) return mk(__uint_as_float(sign), 0.0f);  // +-0
  return mk(__double2float_rn(x), 0.0f);
}

// back to FP64 (two conversions and one add)
__device__ __forceinline__ double dd_join(dd x) { return (double)x.hi + (double)x.lo; }

// rounded to float
__device__ __forceinline__ float dd_float(dd x) { return x.hi + x.lo; }

__device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

// x < y, for normalised pairs
__device__ __forceinline__ bool dd_lt(dd x, dd y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
__device__ __forceinline__ bool dd_neg_p(dd x) { return x.hi < 0.0f; }

inline dd host_split(double x) {
  dd r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}

// host-side split of the constants a kernel needs
struct DDPhys {
  dd a, xi;
  dd ts, tr, ds;                 // theta_s, theta_r, theta_s - theta_r
  dd p1, p2, p3, p4;             // uniform soil parameters
  dd h1, h2, h3, h4, r12, r34;   // sink thresholds, 1/(h1 - h2), 1/(h3 - h4)
  int sink;
};

inline DDPhys make_ddphys(const Phys<double>& P) {
  DDPhys Q;
  Q.a = host_split(P.a);
  Q.xi = host_split(P.xi);
  Q.ts = host_split(P.ts);
  Q.tr = host_split(P.tr);
  Q.ds = host_split(P.ts - P.tr);
  Q.p1 = host_split(P.p1);
  Q.p2 = host_split(P.p2);
  Q.p3 = host_split(P.p3);
  Q.p4 = host_split(P.p4);
  Q.h1 = host_split(P.h1);
  Q.h2 = host_split(P.h2);
  Q.h3 = host_split(P.h3);
  Q.h4 = host_split(P.h4);
  Q.r12 = host_split(P.h1 != P.h2 ? 1.0 / (P.h1 - P.h2) : 0.0);
  Q.r34 = host_split(P.h3 != P.h4 ? 1.0 / (P.h3 - P.h4) : 0.0);
  Q.sink = P.sink;
  return Q;
}

// float-float copy of one material of a layered soil (MatLaw<double>)
struct DDMat {
  int model;
  dd ts, tr, ds, p3, p4;
};

inline DDMat make_ddmat(const MatLaw<double>& M) {
  DDMat D;
  D.model = M.model;
  D.ts = host_split(M.ts);
  D.tr = host_split(M.tr);
  D.ds = host_split(M.ts - M.tr);
  D.p3 = host_split(M.p3);
  D.p4 = host_split(M.p4);
  return D;
}

// with_law for the float-float kernels: fn(LawTag<law>{}, phys, ddphys) with
// both records carrying the cell's theta_s, theta_r, p3, p4
template <int MODEL, typename Fn>
__device__ __forceinline__ auto with_law_dd(const Phys<double>& P, const DDPhys& Q, unsigned m, Fn&& fn) {
  if constexpr (MODEL == COMPOSITE) {
    const MatLaw<double>* __restrict__ M = P.mats + m;
    const DDMat* __restrict__ D = P.ddmats + m;
    Phys<double> Pc = P;
    Pc.ts = M->ts;
    Pc.tr = M->tr;
    Pc.p3 = M->p3;
    Pc.p4 = M->p4;
    DDPhys Qc = Q;
    Qc.ts = D->ts;
    Qc.tr = D->tr;
    Qc.ds = D->ds;
    Qc.p3 = D->p3;
    Qc.p4 = D->p4;
    const int law = D->model;
    if (law == HAVERKAMP) return fn(LawTag<HAVERKAMP>{}, (const Phys<double>&)Pc, (const DDPhys&)Qc);
    if (law == GARDNER) return fn(LawTag<GARDNER>{}, (const Phys<double>&)Pc, (const DDPhys&)Qc);
    return fn(LawTag<VANGENUCHTEN>{}, (const Phys<double>&)Pc, (const DDPhys&)Qc);
  } else {
    return fn(LawTag<MODEL>{}, P, Q);
  }
}

// the same split on the device (per-column soil parameters)
__device__ __forceinline__ DDPhys make_ddphys_dev(const Phys<double>& P) {
  DDPhys Q;
  Q.a = dd_split(P.a);
  Q.xi = dd_split(P.xi);
  Q.ts = dd_split(P.ts);
  Q.tr = dd_split(P.tr);
  Q.ds = dd_split(P.ts - P.tr);
  Q.p1 = dd_split(P.p1);
  Q.p2 = dd_split(P.p2);
  Q.p3 = dd_split(P.p3);
  Q.p4 = dd_split(P.p4);
  Q.h1 = dd_split(P.h1);
  Q.h2 = dd_split(P.h2);
  Q.h3 = dd_split(P.h3);
  Q.h4 = dd_split(P.h4);
  Q.r12 = dd_split(P.h1 != P.h2 ? 1.0 / (P.h1 - P.h2) : 0.0);
  Q.r34 = dd_split(P.h3 != P.h4 ? 1.0 / (P.h3 - P.h4) : 0.0);
  Q.sink = P.sink;
  return Q;
}

// ---------------------------------------------------------------------------
// Constitutive laws (Table 1) in float-float; same branches as law_d/cond_d.
// Arguments outside the float range the routines are written for (a log of
// a value outside [1e-30, 1e30], an exponent beyond +-DD_EXP_MAX) take the
// FP64 routine instead; those are the far dry or far wet tails, where the
// results are at or below 1e-26 of theta_s - theta_r or of Ks.
// ---------------------------------------------------------------------------
#define DD_EXP_MAX 60.0f

__device__ __forceinline__ bool dd_log_ok(dd x) { return x.hi > 1e-30f && x.hi < 1e30f; }
__device__ __forceinline__ bool dd_exp_ok(dd x) { return fabsf(x.hi) <= DD_EXP_MAX; }

// van Genuchten m = 1 - 1/n
__device__ __forceinline__ dd vg_m(dd n) { return dd_sub(mk(1.0f), dd_recip(n)); }

template <int MODEL>
__device__ __forceinline__ dd theta_x(dd psi, dd p1, dd p2, const DDPhys& Q, const Phys<double>& P) {
  if (!dd_neg_p(psi)) return Q.ts;
  const dd h = dd_neg(psi);
  if (MODEL == HAVERKAMP) {                     // theta_r + alpha ds / (alpha + h^beta)
    if (dd_log_ok(h)) {
      const dd e = dd_mul(dd_log(h), p2);
      if (dd_exp_ok(e)) return dd_add(Q.tr, dd_mul(dd_mul(p1, Q.ds), dd_recip(dd_add(p1, dd_exp(e)))));
    }
  } else if (MODEL == GARDNER) {                // theta_r + ds e^{alpha psi}
    const dd e = dd_mul(p1, psi);
    if (dd_exp_ok(e)) return dd_add(Q.tr, dd_mul(Q.ds, dd_exp(e)));
  } else {                                      // theta_r + ds (1 + t)^-m, t = (alpha h)^n
    const dd ah = dd_mul(p1, h);
    if (dd_log_ok(ah)) {
      const dd lt = dd_mul(dd_log(ah), p2);
      if (dd_exp_ok(lt)) {
        const dd e = dd_neg(dd_mul(dd_log1p(dd_exp(lt)), vg_m(p2)));
        if (dd_exp_ok(e)) return dd_add(Q.tr, dd_mul(Q.ds, dd_exp(e)));
      }
    }
  }
  return dd_split(theta_only_d<MODEL>(dd_join(psi), dd_join(p1), dd_join(p2), P));
}

template <int MODEL>
__device__ __forceinline__ dd cond_x(dd psi, dd p1, dd p2, dd Ks, const DDPhys& Q, const Phys<double>& P) {
  if (!dd_neg_p(psi)) return Ks;
  const dd h = dd_neg(psi);
  if (MODEL == HAVERKAMP) {                     // Ks A / (A + h^gamma)
    if (dd_log_ok(h)) {
      const dd e = dd_mul(dd_log(h), Q.p4);
      if (dd_exp_ok(e)) return dd_mul(dd_mul(Ks, Q.p3), dd_recip(dd_add(Q.p3, dd_exp(e))));
    }
  } else if (MODEL == GARDNER) {                // Ks e^{alpha psi}
    const dd e = dd_mul(p1, psi);
    if (dd_exp_ok(e)) return dd_mul(Ks, dd_exp(e));
  } else {                                      // Ks Se^l (1 - (1 - Se^{1/m})^m)^2
    const dd ah = dd_mul(p1, h);
    if (dd_log_ok(ah)) {
      const dd m = vg_m(p2);
      const dd lt = dd_mul(dd_log(ah), p2);     // log t
      if (dd_exp_ok(lt)) {
        const dd t = dd_exp(lt);
        const dd L1 = dd_log1p(t);              // log(1 + t)
        const dd eK = dd_neg(dd_mul(dd_mul(L1, Q.p3), m));
        if (dd_exp_ok(eK)) {
          // log(t / (1 + t)) without cancellation; inner = 1 - (t/(1+t))^m
          const dd lr = t.hi > 1.0f ? dd_neg(dd_log1p(dd_recip(t))) : dd_sub(lt, L1);
          const dd inner = dd_neg(dd_expm1(dd_mul(lr, m)));
          return dd_mul(dd_mul(Ks, dd_exp(eK)), dd_mul(inner, inner));
        }
      }
    }
  }
  return dd_split(cond_d<MODEL>(dd_join(psi), dd_join(p1), dd_join(p2), dd_join(Ks), P));
}

// double in, double out (richards_soil_eval)
template <int MODEL>
__device__ __forceinline__ double theta_dd(double psi, double p1, double p2, const DDPhys& Q,
                                           const Phys<double>& P) {
  return dd_join(theta_x<MODEL>(dd_split(psi), dd_split(p1), dd_split(p2), Q, P));
}
template <int MODEL>
__device__ __forceinline__ double cond_dd(double psi, double p1, double p2, double Ks, const DDPhys& Q,
                                          const Phys<double>& P) {
  return dd_join(cond_x<MODEL>(dd_split(psi), dd_split(p1), dd_split(p2), dd_split(Ks), Q, P));
}

// Feddes sink S = smax alpha_F(psi) (same pieces as feddes()); thresholds
// are compared in float-float, so a psi within 2^-46 of a kink may take the
// neighbouring piece, where alpha_F agrees to that order (it is continuous)
__device__ __forceinline__ dd sink_x(dd psi, dd smax, const DDPhys& Q) {
  if (!Q.sink || !(smax.hi > 0.0f)) return mk(0.0f);
  if (!dd_lt(psi, Q.h1) || dd_lt(psi, Q.h4)) return mk(0.0f);
  if (!dd_lt(psi, Q.h2)) return dd_mul(smax, dd_mul(dd_sub(Q.h1, psi), Q.r12));
  if (!dd_lt(psi, Q.h3)) return smax;
  return dd_mul(smax, dd_mul(dd_sub(psi, Q.h4), Q.r34));
}

}  // namespace rich
