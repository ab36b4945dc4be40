// Device building blocks of the NGS-FAS solver: constitutive laws, the
// conservative 7-point (2d+1) stencil, the bracketed Newton point update,
// the nonlinear defect, and the transfer operators.  Grid kernels and the
// single-block coarse tail both call these functions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fp64math.cuh"

namespace rich {

// COMPOSITE: a layered soil (Section 4.1's composite law, Section 4.2's two
// layers); every cell takes the law of its own material.
enum { HAVERKAMP = 0, GARDNER = 1, VANGENUCHTEN = 2, COMPOSITE = 3 };
constexpr int MAXMAT = 8;      // materials of a layered soil

// FORM_DIRECT: the unknown is psi (eq. point-update as written).
// FORM_DELTA:  the unknown is the correction delta to a frozen psi0, and the
//              storage/sink terms are the increments theta(psi0+delta) -
//              theta(psi0), S(psi0+delta) - S(psi0) evaluated without
//              cancellation (the FP32 inner problem of the mixed mode).
enum { FORM_DIRECT = 0, FORM_DELTA = 1 };

constexpr int RMAX = 6;     // max fine cells per coarse cell along one axis

template <typename T>
struct Level {
  int dim, n0, n1, n2;
  long long ncell;
  T ih2[3];                      // 1/h^2 per axis (0 on unused axes)
  T *u, *ubar, *g, *d;           // iterate, FAS restricted iterate, right side, defect
  const T *Kc, *p1, *p2, *smax;  // lagged conductivity, soil params (nullable), sink coef (nullable)
  const T *psi0;                 // FORM_DELTA: frozen state
  const T *kb[6];                // boundary face conductances (per face cell)
  const uint8_t *mat;            // COMPOSITE: material of each cell of this level
  int cs;                        // 1: g, psi0, p1, p2, smax in the colour-split layout (pix)
};

// Index of cell (i0, i1, i2) (flat index i) in the per-cell parameter arrays
// g, psi0, p1, p2, smax of a level.  Natural layout: i.  Colour-split layout
// (big FP32 levels with an even n0): the cells of each colour packed row by
// row, (i0 >> 1) + n0/2 (i1 + n1 i2), the black half after the red one, so a
// half-sweep reads only its own colour's sectors of these arrays.  u, Kc and
// d keep the natural layout (the stencil reads both colours of them).
__host__ __device__ __forceinline__ unsigned pix_of(int cs, int n0, int n1, int n2, unsigned i, int i0, int i1,
                                                    int i2) {
  if (!cs) return i;
  const unsigned nh = (unsigned)n0 >> 1;
  const unsigned q = (unsigned)(i0 >> 1) + nh * ((unsigned)i1 + (unsigned)n1 * (unsigned)i2);
  return ((i0 + i1 + i2) & 1) ? q + nh * (unsigned)n1 * (unsigned)n2 : q;
}
template <typename T>
__device__ __forceinline__ unsigned pix(const Level<T>& L, long long i, int i0, int i1, int i2) {
  return pix_of(L.cs, L.n0, L.n1, L.n2, (unsigned)i, i0, i1, i2);
}

// One material of a layered soil: its law and the parameters that are not
// per-cell arrays (p1 and p2 are: the level's p1/p2 hold each cell's
// material values on every level).
template <typename T>
struct MatLaw {
  int model;
  T ts, tr, p3, p4;
};

struct DDMat;                    // float-float copy of a MatLaw (ddmath.cuh)

template <typename T>
struct Phys {
  T a, xi, kappa;
  T ts, tr;                      // theta_s, theta_r
  T p1, p2, p3, p4;              // scalar soil parameters
  T h1, h2, h3, h4;              // sink thresholds
  int newton_k;                  // > 0: fixed steps; 0: to round-off
  int sink;
  int lag;                       // BDF2: 1 lags K and the xi term at psi^n, 0 at 2 psi^n - psi^(n-1)
  const MatLaw<T> *mats;         // COMPOSITE: material table (device, MAXMAT entries at most)
  const DDMat *ddmats;           // COMPOSITE, float-float outer layer: the same table as pairs
};

template <int M>
using LawTag = std::integral_constant<int, M>;

// Calls fn(LawTag<law>{}, phys) with the law of a cell and the physics
// record that carries its theta_s, theta_r, p3, p4: MODEL and P themselves,
// or, for a layered soil (MODEL == COMPOSITE), the law and parameters of
// material m.  Cells of one warp with different laws take the branches in turn.
template <int MODEL, typename T, typename Fn>
__device__ __forceinline__ auto with_law(const Phys<T>& P, unsigned m, Fn&& fn) {
  if constexpr (MODEL == COMPOSITE) {
    const MatLaw<T>* __restrict__ M = P.mats + m;
    Phys<T> Q = P;
    Q.ts = M->ts;
    Q.tr = M->tr;
    Q.p3 = M->p3;
    Q.p4 = M->p4;
    const int law = M->model;
    if (law == HAVERKAMP) return fn(LawTag<HAVERKAMP>{}, (const Phys<T>&)Q);
    if (law == GARDNER) return fn(LawTag<GARDNER>{}, (const Phys<T>&)Q);
    return fn(LawTag<VANGENUCHTEN>{}, (const Phys<T>&)Q);
  } else {
    return fn(LawTag<MODEL>{}, P);
  }
}

// material index of cell i (0, and no load, when the soil is not layered)
template <int MODEL>
__device__ __forceinline__ unsigned mat_at(const uint8_t* __restrict__ mat, long long i) {
  if constexpr (MODEL == COMPOSITE) return mat[i];
  else return 0u;
}
template <int MODEL, typename T>
__device__ __forceinline__ unsigned mat_of(const Level<T>& L, long long i) {
  return mat_at<MODEL>(L.mat, i);
}

template <typename T>
struct Xfer {                    // fine level -> next coarser level
  const int *pc[3];              // fine i: number of coarse contributors (1 or 2)
  const int *pj[3];              // fine i: coarse indices [2 i + k]
  const T *pw[3];                // fine i: weights [2 i + k]
  const int *rc[3];              // coarse J: number of fine contributors
  const int *ri[3];              // coarse J: fine indices [RMAX J + k]
  const T *rw[3];                // coarse J: normalised weights
};

// ---------------------------------------------------------------------------
// Constitutive laws (Table 1 of the paper); psi >= 0 gives theta_s, Ks and a
// zero capacity for all three laws.
// ---------------------------------------------------------------------------
template <int MODEL>
__device__ __forceinline__ void law_d(double psi, double p1, double p2, const Phys<double>& P,
                                      double& th, double& dth) {
  if (!(psi < 0.0)) { th = P.ts; dth = 0.0; return; }
  const double h = -psi, ds = P.ts - P.tr;
  if (MODEL == HAVERKAMP) {
    // theta = theta_r + alpha ds / (alpha + h^beta)
    const double u = fx::exp(p2 * fx::log(h));
    const double den = p1 + u;
    th = P.tr + p1 * ds / den;
    dth = p1 * ds * p2 * (u / h) / (den * den);
  } else if (MODEL == GARDNER) {
    const double e = fx::exp(p1 * psi);
    th = P.tr + ds * e;
    dth = p1 * ds * e;
  } else {
    // Se = (1 + t)^-m, t = (alpha h)^n, m = 1 - 1/n
    const double n = p2, m = 1.0 - 1.0 / n;
    const double t = fx::exp(n * fx::log(p1 * h));
    const double Se = fx::exp(-m * fx::log1p(t));
    th = P.tr + ds * Se;
    dth = ds * m * n * (t / h) * Se / (1.0 + t);
  }
}

template <int MODEL>
__device__ __forceinline__ double theta_only_dm(double psi, double p1, double p2, double m, const Phys<double>& P) {
  if (!(psi < 0.0)) return P.ts;
  const double h = -psi, ds = P.ts - P.tr;
  if (MODEL == HAVERKAMP) return P.tr + p1 * ds / (p1 + fx::exp(p2 * fx::log(h)));
  if (MODEL == GARDNER) return P.tr + ds * fx::exp(p1 * psi);
  const double n = p2;
  return P.tr + ds * fx::exp(-m * fx::log1p(fx::exp(n * fx::log(p1 * h))));
}

// van Genuchten's m = 1 - 1/n (kernels that evaluate the laws of a per-cell
// n field read it from a copy made with this same expression)
__device__ __forceinline__ double vg_m(double n) { return 1.0 - 1.0 / n; }

// theta of one law; m (van Genuchten only) from n
template <int MODEL>
__device__ __forceinline__ double theta_only_d(double psi, double p1, double p2, const Phys<double>& P) {
  return theta_only_dm<MODEL>(psi, p1, p2, (MODEL == VANGENUCHTEN && psi < 0.0) ? vg_m(p2) : 0.0, P);
}

// Hydraulic conductivity.  For van Genuchten-Mualem, Se^{1/m} = 1/(1+t), so
// 1 - (1 - Se^{1/m})^m = -expm1(m log(t/(1+t))), evaluated without
// cancellation in both the wet (t < 1) and the dry (t > 1) range.  With
// lt = log t and e = exp(-|lt|) (t when t <= 1, 1/t when t > 1):
//   log(1 + t)       = log1p(e) + max(lt, 0),
//   log(t / (1 + t)) = min(lt, 0) - log1p(e),
// one exponential and one log1p for both ranges, no division and no branch.
template <int MODEL>
__device__ __forceinline__ double cond_dm(double psi, double p1, double p2, double m, double Ks,
                                          const Phys<double>& P) {
  if (!(psi < 0.0)) return Ks;
  const double h = -psi;
  if (MODEL == HAVERKAMP) return Ks * P.p3 / (P.p3 + fx::exp(P.p4 * fx::log(h)));
  if (MODEL == GARDNER) return Ks * fx::exp(p1 * psi);
  const double n = p2;
  const double lt = n * fx::log(p1 * h);
  const double l1 = fx::log1p(fx::exp(-fabs(lt)));
  const double L1 = l1 + fmax(lt, 0.0);
  const double lr = fmin(lt, 0.0) - l1;
  const double inner = -fx::expm1(m * lr);
  return Ks * fx::exp(-P.p3 * m * L1) * inner * inner;
}

template <int MODEL>
__device__ __forceinline__ double cond_d(double psi, double p1, double p2, double Ks, const Phys<double>& P) {
  return cond_dm<MODEL>(psi, p1, p2, (MODEL == VANGENUCHTEN && psi < 0.0) ? vg_m(p2) : 0.0, Ks, P);
}

__device__ __forceinline__ double cond_model_d(int model, double psi, double p1, double p2,
                                               double Ks, const Phys<double>& P) {
  if (model == HAVERKAMP) return cond_d<HAVERKAMP>(psi, p1, p2, Ks, P);
  if (model == GARDNER) return cond_d<GARDNER>(psi, p1, p2, Ks, P);
  return cond_d<VANGENUCHTEN>(psi, p1, p2, Ks, P);
}
__device__ __forceinline__ double theta_model_d(int model, double psi, double p1, double p2,
                                                const Phys<double>& P) {
  if (model == HAVERKAMP) return theta_only_d<HAVERKAMP>(psi, p1, p2, P);
  if (model == GARDNER) return theta_only_d<GARDNER>(psi, p1, p2, P);
  return theta_only_d<VANGENUCHTEN>(psi, p1, p2, P);
}

// Increment form in FP32: Dth = theta(psi0 + x) - theta(psi0) and
// dth = theta'(psi0 + x), with the differences taken through expm1/log1p of
// the ratio (psi0 + x)/psi0, so that Dth is accurate relative to itself.
template <int MODEL>
__device__ __forceinline__ void dlaw_f(float psi0, float x, float p1, float p2, const Phys<float>& P,
                                       float& Dth, float& dth) {
  const float ds = P.ts - P.tr;
  const float psi1 = psi0 + x;
  const bool wet0 = !(psi0 < 0.0f), wet1 = !(psi1 < 0.0f);
  if (MODEL == GARDNER) {
    const float al = p1;
    if (!wet0) {
      const float e0 = expf(al * psi0);
      if (!wet1) {
        const float em = expm1f(al * x);
        Dth = ds * e0 * em;
        dth = al * ds * e0 * (1.0f + em);
      } else {
        Dth = -ds * expm1f(al * psi0);
        dth = 0.0f;
      }
    } else if (!wet1) {
      Dth = ds * expm1f(al * psi1);
      dth = al * ds * expf(al * psi1);
    } else {
      Dth = 0.0f; dth = 0.0f;
    }
  } else if (MODEL == HAVERKAMP) {
    const float al = p1, be = p2;
    if (!wet0) {
      const float h0 = -psi0;
      const float u0 = expf(be * logf(h0));
      if (!wet1) {
        const float du = u0 * expm1f(be * log1pf(x / psi0));
        const float u1 = u0 + du, h1 = -psi1;
        const float den1 = al + u1;
        Dth = -al * ds * du / ((al + u0) * den1);
        dth = al * ds * be * (u1 / h1) / (den1 * den1);
      } else {
        Dth = ds * u0 / (al + u0);
        dth = 0.0f;
      }
    } else if (!wet1) {
      const float h1 = -psi1;
      const float u1 = expf(be * logf(h1));
      const float den1 = al + u1;
      Dth = -ds * u1 / den1;
      dth = al * ds * be * (u1 / h1) / (den1 * den1);
    } else {
      Dth = 0.0f; dth = 0.0f;
    }
  } else {
    const float al = p1, n = p2, m = 1.0f - 1.0f / n;
    if (!wet0) {
      const float h0 = -psi0;
      const float t0 = expf(n * logf(al * h0));
      const float L0 = log1pf(t0);
      const float Se0 = expf(-m * L0);
      if (!wet1) {
        const float dt = t0 * expm1f(n * log1pf(x / psi0));      // t1 - t0
        const float t1 = t0 + dt;
        const float dL = log1pf(dt / (1.0f + t0));                // log(1+t1) - log(1+t0)
        const float dSe = Se0 * expm1f(-m * dL);
        const float Se1 = Se0 + dSe;
        Dth = ds * dSe;
        dth = ds * m * n * (t1 / (-psi1)) * Se1 / (1.0f + t1);
      } else {
        Dth = -ds * expm1f(-m * L0);
        dth = 0.0f;
      }
    } else if (!wet1) {
      const float h1 = -psi1;
      const float t1 = expf(n * logf(al * h1));
      const float L1 = log1pf(t1);
      Dth = ds * expm1f(-m * L1);
      dth = ds * m * n * (t1 / h1) * expf(-m * L1) / (1.0f + t1);
    } else {
      Dth = 0.0f; dth = 0.0f;
    }
  }
}

// ---------------------------------------------------------------------------
// Fast single-precision pieces for the inner correction problem.  The inner
// FP32 solve only has to be accurate to ~1e-5 relative (the float-float outer
// defect correction removes the rest), but the increments must stay free of
// cancellation: log1p and expm1 of small arguments come from their Taylor
// series (truncation below 1e-10 relative for |x| < 1/32), larger arguments
// use the hardware approximations __logf / __expf (relative error ~1e-6 of a
// result that is then not small).
// ---------------------------------------------------------------------------
// (both forms are evaluated and one is selected: no branch, so lanes of a
// warp on either side of 1/32 do not split it into two passes)
__device__ __forceinline__ float fast_log1p(float x) {
  // x - x^2/2 + x^3/3 - x^4/4 + x^5/5 - x^6/6
  const float p = fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, -1.0f / 6.0f, 0.2f), -0.25f), 1.0f / 3.0f), -0.5f), 1.0f);
  const float big = __logf(1.0f + x);
  return fabsf(x) < 0.03125f ? x * p : big;
}

__device__ __forceinline__ float fast_expm1(float x) {
  // x + x^2/2 + x^3/6 + x^4/24 + x^5/120 + x^6/720
  const float p = fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.0f / 720.0f, 1.0f / 120.0f), 1.0f / 24.0f),
                                           1.0f / 6.0f), 0.5f), 1.0f);
  const float big = __expf(x) - 1.0f;
  return fabsf(x) < 0.03125f ? x * p : big;
}

// Same increments as dlaw_f, built from the fast pieces above, split into
// the part that depends on psi0 only (once per point update) and the part
// that depends on the correction x (once per Newton step).
struct DBase {
  float psi0, inv_psi0;
  bool wet0;
  float a0, b0, c0;      // VG: t0, log1p(t0), Se0; Haverkamp: u0, log(u0); Gardner: e0
  float m;               // VG: 1 - 1/n
};

// Largest exponent a power t = (alpha h)^n or u = h^beta of a trial state may
// reach (e^80 ~ 5.5e34, below FLT_MAX with room for 1 + t and products).  A
// bracketed point solve on a coarse level with a tiny coupling can probe
// heads of -1e6 m and beyond, where the power would overflow and its ratios
// turn into inf/inf; there theta = theta_r and theta' = 0 to far below FP32
// resolution either way, so capping the exponent changes nothing else.
constexpr float POW_EXP_MAX = 80.0f;

template <int MODEL>
__device__ __forceinline__ DBase dbase(float psi0, float p1, float p2) {
  DBase B;
  B.psi0 = psi0;
  B.wet0 = !(psi0 < 0.0f);
  B.inv_psi0 = B.wet0 ? 0.0f : __fdividef(1.0f, psi0);
  B.a0 = B.b0 = B.c0 = 0.0f;
  B.m = MODEL == VANGENUCHTEN ? 1.0f - __fdividef(1.0f, p2) : 0.0f;
  if (!B.wet0) {
    if (MODEL == GARDNER) {
      B.a0 = __expf(p1 * psi0);
    } else if (MODEL == HAVERKAMP) {
      const float lu = fminf(p2 * __logf(-psi0), POW_EXP_MAX);   // h0^beta through the hardware log/exp
      B.a0 = __expf(lu);
      B.b0 = lu;
    } else {
      const float m = B.m;
      B.a0 = __expf(fminf(p2 * __logf(p1 * -psi0), POW_EXP_MAX));   // (alpha h0)^n
      B.b0 = fast_log1p(B.a0);
      B.c0 = __expf(-m * B.b0);
    }
  }
  return B;
}

template <int MODEL>
__device__ __forceinline__ void dincr(const DBase& B, float x, float p1, float p2, const Phys<float>& P,
                                      float& Dth, float& dth) {
  const float ds = P.ts - P.tr;
  const float psi1 = B.psi0 + x;
  const bool wet1 = !(psi1 < 0.0f);
  if (MODEL == GARDNER) {
    const float al = p1;
    if (!B.wet0) {
      const float e0 = B.a0;
      if (!wet1) {
        const float em = fast_expm1(al * x);
        Dth = ds * e0 * em;
        dth = al * ds * e0 * (1.0f + em);
      } else {
        Dth = -ds * fast_expm1(al * B.psi0);
        dth = 0.0f;
      }
    } else if (!wet1) {
      Dth = ds * fast_expm1(al * psi1);
      dth = al * ds * __expf(al * psi1);
    } else {
      Dth = 0.0f; dth = 0.0f;
    }
  } else if (MODEL == HAVERKAMP) {
    const float al = p1, be = p2;
    if (!B.wet0) {
      const float u0 = B.a0;
      if (!wet1) {
        // (u1 = u0 (psi1/psi0)^beta, its exponent capped as in dbase)
        // (psi1/psi0 > 0 here; its rounded value is kept above 2^-24)
        const float q = fmaxf(x * B.inv_psi0, -0.99999994f);
        const float du = u0 * fast_expm1(fminf(be * fast_log1p(q), POW_EXP_MAX - B.b0));
        const float u1 = u0 + du, h1 = -psi1;
        const float den1 = al + u1;
        Dth = __fdividef(-al * ds * du, (al + u0) * den1);
        dth = __fdividef(al * ds * be * __fdividef(u1, h1), den1 * den1);
      } else {
        Dth = __fdividef(ds * u0, al + u0);
        dth = 0.0f;
      }
    } else if (!wet1) {
      const float h1 = -psi1;
      const float u1 = __expf(fminf(be * __logf(h1), POW_EXP_MAX));
      const float den1 = al + u1;
      Dth = __fdividef(-ds * u1, den1);
      dth = __fdividef(al * ds * be * __fdividef(u1, h1), den1 * den1);
    } else {
      Dth = 0.0f; dth = 0.0f;
    }
  } else {
    const float al = p1, n = p2, m = B.m;
    if (!B.wet0) {
      const float t0 = B.a0, L0 = B.b0, Se0 = B.c0;
      if (!wet1) {
        // (t1 = t0 (psi1/psi0)^n, its exponent capped as in dbase)
        const float q = fmaxf(x * B.inv_psi0, -0.99999994f);     // (as for Haverkamp)
        const float dt = t0 * fast_expm1(fminf(n * fast_log1p(q), POW_EXP_MAX - B.b0));
        const float t1 = t0 + dt;
        const float dSe = Se0 * fast_expm1(-m * fast_log1p(__fdividef(dt, 1.0f + t0)));
        const float Se1 = Se0 + dSe;
        Dth = ds * dSe;
        dth = ds * m * n * __fdividef(t1, -psi1) * __fdividef(Se1, 1.0f + t1);
      } else {
        Dth = -ds * fast_expm1(-m * L0);
        dth = 0.0f;
      }
    } else if (!wet1) {
      const float h1 = -psi1;
      const float t1 = __expf(fminf(n * __logf(al * h1), POW_EXP_MAX));
      const float L1 = fast_log1p(t1);
      Dth = ds * fast_expm1(-m * L1);
      dth = ds * m * n * __fdividef(t1, h1) * __fdividef(__expf(-m * L1), 1.0f + t1);
    } else {
      Dth = 0.0f; dth = 0.0f;
    }
  }
}

template <int MODEL>
__device__ __forceinline__ void dlaw_fast(float psi0, float x, float p1, float p2, const Phys<float>& P,
                                          float& Dth, float& dth) {
  dincr<MODEL>(dbase<MODEL>(psi0, p1, p2), x, p1, p2, P, Dth, dth);
}

// ---------------------------------------------------------------------------
// Sink reading: S = smax * alpha_F(psi), alpha_F piecewise linear through
// (h4,0), (h3,1), (h2,1), (h1,0), zero outside; right derivatives at kinks.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int feddes(T psi, const Phys<T>& P, T& a, T& da) {
  if (psi >= P.h1) { a = T(0); da = T(0); return 0; }
  if (psi < P.h4) { a = T(0); da = T(0); return 4; }
  if (psi >= P.h2) { a = (P.h1 - psi) / (P.h1 - P.h2); da = T(-1) / (P.h1 - P.h2); return 1; }
  if (psi >= P.h3) { a = T(1); da = T(0); return 2; }
  a = (psi - P.h4) / (P.h3 - P.h4); da = T(1) / (P.h3 - P.h4); return 3;
}

template <typename T>
__device__ __forceinline__ void sink_direct(T psi, T smax, const Phys<T>& P, T& S, T& dS) {
  T a = T(0), da = T(0);
  if (P.sink && smax > T(0)) feddes(psi, P, a, da);
  S = a * smax;
  dS = da * smax;
}

// S(psi0 + x) - S(psi0): exact slope * x on a common linear piece.
template <typename T>
__device__ __forceinline__ void sink_delta(T psi0, T x, T smax, const Phys<T>& P, T& DS, T& dS) {
  if (!(P.sink && smax > T(0))) { DS = T(0); dS = T(0); return; }
  T a0, da0, a1, da1;
  const int k0 = feddes(psi0, P, a0, da0);
  const int k1 = feddes(psi0 + x, P, a1, da1);
  DS = (k0 == k1) ? smax * da1 * x : smax * (a1 - a0);
  dS = smax * da1;
}

// ---------------------------------------------------------------------------
// Stencil: m_ii and sum_j m_ij u_j for cell i (interior faces K_f/h^2 with
// K_f = (Kc_i + Kc_j)/2; Dirichlet faces 2 kb/h^2 on the diagonal).
// ---------------------------------------------------------------------------
// (YZI: the caller knows that the cell of a 3-d level is interior along axes
// 1 and 2, so only axis 0 is tested for boundary faces)
template <typename T, bool YZI = false>
__device__ __forceinline__ void stencil(const Level<T>& L, long long i, int i0, int i1, int i2,
                                        const T* __restrict__ u, T& mii, T& off) {
  // neighbours through base pointers and 32-bit strides (levels hold fewer
  // than 2^31 cells)
  const T* __restrict__ Kp = L.Kc + i;
  const T* __restrict__ up = u + i;
  const T Ki = Kp[0];
  T dg = T(0), of = T(0);
  // K_f / h^2 = (Kc_i + Kc_j) * (s/2): halving s is exact, so this equals
  // ((Kc_i + Kc_j) / 2) * s bit for bit
  {
    const T s = L.ih2[0], hs = T(0.5) * s;
    if (i0 > 0) { const T m = (Ki + Kp[-1]) * hs; dg += m; of += m * up[-1]; }
    else dg += T(2) * L.kb[0][i1 + L.n1 * i2] * s;
    if (i0 < L.n0 - 1) { const T m = (Ki + Kp[1]) * hs; dg += m; of += m * up[1]; }
    else dg += T(2) * L.kb[1][i1 + L.n1 * i2] * s;
  }
  if (YZI) {
    {
      const T s = L.ih2[1], hs = T(0.5) * s;
      const int st = L.n0;
      { const T m = (Ki + Kp[-st]) * hs; dg += m; of += m * up[-st]; }
      { const T m = (Ki + Kp[st]) * hs; dg += m; of += m * up[st]; }
    }
    {
      const T s = L.ih2[2], hs = T(0.5) * s;
      const int st = L.n0 * L.n1;
      { const T m = (Ki + Kp[-st]) * hs; dg += m; of += m * up[-st]; }
      { const T m = (Ki + Kp[st]) * hs; dg += m; of += m * up[st]; }
    }
    mii = dg;
    off = of;
    return;
  }
  if (L.dim > 1) {
    const T s = L.ih2[1], hs = T(0.5) * s;
    const int st = L.n0;
    if (i1 > 0) { const T m = (Ki + Kp[-st]) * hs; dg += m; of += m * up[-st]; }
    else dg += T(2) * L.kb[2][i0 + L.n0 * i2] * s;
    if (i1 < L.n1 - 1) { const T m = (Ki + Kp[st]) * hs; dg += m; of += m * up[st]; }
    else dg += T(2) * L.kb[3][i0 + L.n0 * i2] * s;
  }
  if (L.dim > 2) {
    const T s = L.ih2[2], hs = T(0.5) * s;
    const int st = L.n0 * L.n1;
    if (i2 > 0) { const T m = (Ki + Kp[-st]) * hs; dg += m; of += m * up[-st]; }
    else dg += T(2) * L.kb[4][i0 + L.n0 * i1] * s;
    if (i2 < L.n2 - 1) { const T m = (Ki + Kp[st]) * hs; dg += m; of += m * up[st]; }
    else dg += T(2) * L.kb[5][i0 + L.n0 * i1] * s;
  }
  mii = dg;
  off = of;
}

template <typename T>
__device__ __forceinline__ T tol_of();
template <>
__device__ __forceinline__ double tol_of<double>() { return 1e-15; }
template <>
__device__ __forceinline__ float tol_of<float>() { return 1e-7f; }

// Storage + sink part and its derivative at x for either form.
template <typename T, int FORM, int MODEL>
__device__ __forceinline__ void storage(T x, T psi0, T p1, T p2, T smax, const Phys<T>& P,
                                        T& val, T& der) {
  if constexpr (FORM == FORM_DIRECT) {
    static_assert(sizeof(T) == 8, "direct form is FP64");
    double th, dth, S, dS;
    law_d<MODEL>(x, p1, p2, P, th, dth);
    sink_direct(x, smax, P, S, dS);
    val = P.a * th + S;
    der = P.a * dth + dS;
  } else {
    static_assert(sizeof(T) == 4, "increment form is FP32");
    float Dth, dth, DS, dS;
    dlaw_fast<MODEL>(psi0, x, p1, p2, P, Dth, dth);
    sink_delta(psi0, x, smax, P, DS, dS);
    val = P.a * Dth + DS;
    der = P.a * dth + dS;
  }
}

// Scalar solve of  storage(x) + cc x = f  (eq. point-update).  The left side
// increases strictly (cc > 0), the root lies in [lo, hi]; Newton from x0,
// bisection whenever a step leaves the current bracket.
// NK > 0: exactly NK steps fixed at compile time (must equal P.newton_k);
// NK = 0: P.newton_k steps (0: to round-off).
// FP32 increment form with a fixed step count: a solve does not end on a
// bisection.  Where the coupling is tiny (dry cells of a steep law on a
// coarse level) the bracket spans millions of metres and its midpoint is no
// estimate of the root; after a bisection up to BISECT_EXTRA further steps
// run until one is a Newton step inside the bracket.  Solves that never
// bisect take exactly the fixed count, as before.
constexpr int BISECT_EXTRA = 12;

template <typename T, int FORM, int MODEL, int NK = 0>
__device__ __forceinline__ T point_solve(T cc, T f, T x0, T psi0, T p1, T p2, T smax,
                                         const Phys<T>& P) {
  if (!(cc > T(0))) {
    // no coupling and no shift (c = 0): shift kappa (x - x0), kappa = 1e-6 a,
    // which keeps the root and provides the bracket
    const T k = T(1e-6) * P.a;
    f += (k - cc) * x0;
    cc = k;
  }
  const T ds = P.ts - P.tr;
  T lo, hi;
  if constexpr (FORM == FORM_DIRECT) {
    lo = (f - P.a * P.ts - smax) / cc;
    hi = (f - P.a * P.tr) / cc;
  } else {
    // FP32: both ends through one approximate reciprocal; each end has a
    // slack of (a ds + smax)/cc beyond the root, far above its 2^-22 error
    const T rc = __fdividef(1.0f, cc);
    lo = (f - P.a * ds - smax) * rc;
    hi = (f + P.a * ds + smax) * rc;
  }
  T x = x0 < lo ? lo : (x0 > hi ? hi : x0);
  const int maxit = NK > 0 ? NK : (P.newton_k > 0 ? P.newton_k : 200);
  DBase B;
  T sa0 = T(0), sda0 = T(0);
  int sk0 = 0;
  if constexpr (FORM == FORM_DELTA) {
    B = dbase<MODEL>(psi0, p1, p2);
    if (P.sink && smax > T(0)) sk0 = feddes(psi0, P, sa0, sda0);
  }
  // one safeguarded step; returns true when the solve is done.  *bis: the
  // step was a bisection
  auto step = [&](bool* bis) -> bool {
    *bis = false;
    T val, der;
    if constexpr (FORM == FORM_DELTA) {
      float Dth, dth;
      dincr<MODEL>(B, x, p1, p2, P, Dth, dth);
      T DS = T(0), dS = T(0);
      if (P.sink && smax > T(0)) {
        T a1, da1;
        const int k1 = feddes(psi0 + x, P, a1, da1);
        DS = (k1 == sk0) ? smax * da1 * x : smax * (a1 - sa0);
        dS = smax * da1;
      }
      val = P.a * Dth + DS;
      der = P.a * dth + dS;
    } else {
      storage<T, FORM, MODEL>(x, psi0, p1, p2, smax, P, val, der);
    }
    const T F = val + cc * x - f;
    const T dF = der + cc;
    if (F == T(0)) return true;
    if (F > T(0)) hi = x; else lo = x;
    T xn;
    if constexpr (sizeof(T) == 4) xn = x - __fdividef(F, dF);    // dF > 0; a 2-ulp step error is harmless
    else xn = x - F / dF;
    // a step strictly inside the bracket, or below round-off, is kept;
    // anything else (outside, or onto an end) is replaced by bisection
    const T tiny = tol_of<T>() * (fabs(x) > T(1) ? fabs(x) : T(1));
    if (!(xn > lo && xn < hi) && !(fabs(xn - x) <= tiny)) {
      xn = T(0.5) * (lo + hi);
      *bis = true;
    }
    const T stp = fabs(xn - x);
    x = xn;
    if (NK == 0 && P.newton_k <= 0 && stp <= tiny) return true;
    // FP32 increment form: a step below 2^-20 of |x| leaves nothing for the
    // next one to change at this precision (quadratic convergence)
    if constexpr (FORM == FORM_DELTA) {
      if (stp <= 9.5367431640625e-7f * fabsf(x)) return true;
    }
    return false;
  };
  bool bis = false, done = false;
#pragma unroll(NK > 0 ? NK : 1)
  for (int it = 0; it < maxit; ++it) {
    if (step(&bis)) { done = true; break; }
  }
  if constexpr (FORM == FORM_DELTA) {
    if (P.newton_k > 0 && !done)
      for (int e = 0; e < BISECT_EXTRA && bis; ++e)
        if (step(&bis)) break;
  }
  return x;
}

template <typename T, int FORM, int MODEL, int NK = 0>
__device__ __forceinline__ void point_update(const Level<T>& L, const Phys<T>& P, long long i,
                                             int i0, int i1, int i2) {
  T mii, off;
  stencil(L, i, i0, i1, i2, L.u, mii, off);
  const T ui = L.u[i];
  const T cc = P.xi + P.kappa + mii;
  const unsigned q = pix(L, i, i0, i1, i2);
  const T f = L.g[q] + off + P.kappa * ui;
  const T p1 = L.p1 ? L.p1[q] : P.p1;
  const T p2 = L.p2 ? L.p2[q] : P.p2;
  const T smax = L.smax ? L.smax[q] : T(0);
  const T psi0 = FORM == FORM_DELTA ? L.psi0[q] : T(0);
  L.u[i] = with_law<MODEL>(P, mat_of<MODEL>(L, i), [&](auto law, const Phys<T>& Q) {
    return point_solve<T, FORM, decltype(law)::value, NK>(cc, f, ui, psi0, p1, p2, smax, Q);
  });
}

// Operands of one point update, gathered before any of them is used, so that
// a thread can issue the loads of its next cell before it solves the current
// one (the sweep is bound by load latency, not by bandwidth).  Face f =
// 2 axis + side; on a boundary face Kn holds the face conductance kb; on an
// axis the grid does not have, Kn = un = 0 and 1/h^2 = 0, so m_f = 0.
template <typename T>
struct CellOps {
  unsigned i;
  bool valid;
  unsigned bmask;                // bit f: face f lies on the boundary
  unsigned mat;                  // COMPOSITE: the cell's material
  T ui, Ki, g, psi0, p1, p2, smax;
  T Kn[6], un[6];
};

// YZI: the caller knows that the cell is interior along axes 1 and 2 of a
// 3-d level (no boundary face there), so only axis 0 is tested
template <typename T, int FORM, int MODEL, bool YZI = false>
__device__ __forceinline__ void gather(const Level<T>& L, const Phys<T>& P, int i0, int i1, int i2, CellOps<T>& c) {
  const unsigned i = (unsigned)(i0 + L.n0 * (i1 + L.n1 * i2));
  c.i = i;
  c.mat = mat_of<MODEL>(L, i);
  const T* __restrict__ Kp = L.Kc + i;
  const T* __restrict__ up = L.u + i;
  c.Ki = Kp[0];
  c.ui = up[0];
  const unsigned q = pix(L, i, i0, i1, i2);
  c.g = L.g[q];
  c.psi0 = FORM == FORM_DELTA ? L.psi0[q] : T(0);
  c.p1 = L.p1 ? L.p1[q] : P.p1;
  c.p2 = L.p2 ? L.p2[q] : P.p2;
  c.smax = L.smax ? L.smax[q] : T(0);
  unsigned bm = 0;
  const int ii[3] = {i0, i1, i2};
  const int nn[3] = {L.n0, L.n1, L.n2};
  const int st[3] = {1, L.n0, L.n0 * L.n1};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (YZI && a > 0) {
      c.Kn[2 * a] = Kp[-st[a]]; c.un[2 * a] = up[-st[a]];
      c.Kn[2 * a + 1] = Kp[st[a]]; c.un[2 * a + 1] = up[st[a]];
      continue;
    }
    const int fc = a == 0 ? i1 + L.n1 * i2 : (a == 1 ? i0 + L.n0 * i2 : i0 + L.n0 * i1);
    if (a >= L.dim) {
      c.Kn[2 * a] = c.Kn[2 * a + 1] = T(0);
      c.un[2 * a] = c.un[2 * a + 1] = T(0);
      continue;
    }
    if (ii[a] > 0) { c.Kn[2 * a] = Kp[-st[a]]; c.un[2 * a] = up[-st[a]]; }
    else { c.Kn[2 * a] = L.kb[2 * a][fc]; c.un[2 * a] = T(0); bm |= 1u << (2 * a); }
    if (ii[a] < nn[a] - 1) { c.Kn[2 * a + 1] = Kp[st[a]]; c.un[2 * a + 1] = up[st[a]]; }
    else { c.Kn[2 * a + 1] = L.kb[2 * a + 1][fc]; c.un[2 * a + 1] = T(0); bm |= 1u << (2 * a + 1); }
  }
  c.bmask = bm;
}

// the point update of a gathered cell (same sums, in the same order, as
// stencil() and point_update())
// m_ii (dg) and sum_j m_ij u_j (of) of a gathered cell: the sums of
// stencil(), in its order
template <typename T, bool YZI = false>
__device__ __forceinline__ void cell_sums(const Level<T>& L, const CellOps<T>& c, T& dg, T& of) {
  dg = T(0);
  of = T(0);
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const T s = L.ih2[f >> 1];
    if ((!YZI || f < 2) && (c.bmask & (1u << f))) {
      dg += T(2) * c.Kn[f] * s;
    } else {
      const T m = (c.Ki + c.Kn[f]) * (T(0.5) * s);
      dg += m;
      of += m * c.un[f];
    }
  }
}

// g_i - N(u)_i of a gathered cell at the value x of u_i, with its sums dg, of
// (the expression of apply_N(), so both give the same bits)
template <typename T, int FORM, int MODEL>
__device__ __forceinline__ T cell_defect(const Phys<T>& P, const CellOps<T>& c, T dg, T of, T x) {
  T val, der;
  with_law<MODEL>(P, c.mat, [&](auto law, const Phys<T>& Q) {
    storage<T, FORM, decltype(law)::value>(x, c.psi0, c.p1, c.p2, c.smax, Q, val, der);
    return 0;
  });
  return c.g - (val + P.xi * x + dg * x - of);
}

template <typename T, int FORM, int MODEL, int NK = 0, bool YZI = false>
__device__ __forceinline__ T solve_cell_sums(const Level<T>& L, const Phys<T>& P, const CellOps<T>& c, T dg, T of) {
  const T cc = P.xi + P.kappa + dg;
  const T f = c.g + of + P.kappa * c.ui;
  return with_law<MODEL>(P, c.mat, [&](auto law, const Phys<T>& Q) {
    return point_solve<T, FORM, decltype(law)::value, NK>(cc, f, c.ui, c.psi0, c.p1, c.p2, c.smax, Q);
  });
}

template <typename T, int FORM, int MODEL, int NK = 0, bool YZI = false>
__device__ __forceinline__ T solve_cell(const Level<T>& L, const Phys<T>& P, const CellOps<T>& c) {
  T dg, of;
  cell_sums<T, YZI>(L, c, dg, of);
  return solve_cell_sums<T, FORM, MODEL, NK, YZI>(L, P, c, dg, of);
}

// N(u)_i = storage(u_i) + xi u_i + m_ii u_i - sum_j m_ij u_j   (eq. Nh-def)
template <typename T, int FORM, int MODEL, bool YZI = false>
__device__ __forceinline__ T apply_N(const Level<T>& L, const Phys<T>& P, const T* __restrict__ u,
                                     long long i, int i0, int i1, int i2) {
  T mii, off;
  stencil<T, YZI>(L, i, i0, i1, i2, u, mii, off);
  const unsigned q = pix(L, i, i0, i1, i2);
  const T p1 = L.p1 ? L.p1[q] : P.p1;
  const T p2 = L.p2 ? L.p2[q] : P.p2;
  const T smax = L.smax ? L.smax[q] : T(0);
  const T psi0 = FORM == FORM_DELTA ? L.psi0[q] : T(0);
  T val, der;
  with_law<MODEL>(P, mat_of<MODEL>(L, i), [&](auto law, const Phys<T>& Q) {
    storage<T, FORM, decltype(law)::value>(u[i], psi0, p1, p2, smax, Q, val, der);
    return 0;
  });
  return val + P.xi * u[i] + mii * u[i] - off;
}

// (levels hold fewer than 2^31 cells: 32-bit division suffices)
__device__ __forceinline__ void cell_coords(const int n0, const int n1, long long i, int& i0, int& i1,
                                            int& i2) {
  const unsigned ui = (unsigned)i;
  const unsigned r = ui / (unsigned)n0;
  i0 = (int)(ui - r * (unsigned)n0);
  i1 = (int)(r % (unsigned)n1);
  i2 = (int)(r / (unsigned)n1);
}

// thread index t over one colour -> cell (x pairs, colour chosen per row)
__device__ __forceinline__ bool color_cell(int n0, int n1, long long t, int color, int& i0, int& i1,
                                           int& i2, long long& i) {
  const unsigned nh = (unsigned)((n0 + 1) >> 1);
  const unsigned ut = (unsigned)t;
  const unsigned r = ut / nh;
  const int p = (int)(ut - r * nh);
  i1 = (int)(r % (unsigned)n1);
  i2 = (int)(r / (unsigned)n1);
  i0 = 2 * p + ((color + i1 + i2) & 1);
  if (i0 >= n0) return false;
  i = i0 + (long long)n0 * (i1 + (long long)n1 * i2);
  return true;
}

// ---------------------------------------------------------------------------
// One row of the linear interpolation from a coarse axis (nc cells) to fine
// cell i of a fine axis (nf cells): the coarse coordinate of the fine centre
// is ((2i+1) nc - nf) / (2 nf); a ghost beyond either end folds into the end
// cell with factor slo / shi (+1 constant extrapolation, -1 zero on a
// Dirichlet face).  Entries with zero weight are dropped, equal indices merged.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void interp_row(int nf, int nc, int i, double slo, double shi, int* idx, double* w,
                                           int& cnt) {
  cnt = 0;
  auto add = [&](int j, double wt) {
    if (wt == 0.0) return;
    for (int k = 0; k < cnt; ++k)
      if (idx[k] == j) { w[k] += wt; return; }
    idx[cnt] = j;
    w[cnt] = wt;
    ++cnt;
  };
  if (nf == 1) { add(0, 1.0); return; }
  const long long num = (long long)(2 * i + 1) * nc - nf, den = 2LL * nf;
  const long long J0 = num >= 0 ? num / den : -((-num + den - 1) / den);
  const double wt = (double)(num - J0 * den) / (double)den;
  const long long J1 = J0 + 1;
  if (J0 < 0) add(0, (1.0 - wt) * slo); else add((int)J0, 1.0 - wt);
  if (J1 >= nc) add(nc - 1, wt * shi); else add((int)J1, wt);
}

// ---------------------------------------------------------------------------
// Transfers (restriction: normalised full weighting; prolongation: linear).
// ---------------------------------------------------------------------------
template <typename T>
// (cs: fine is a per-cell parameter array of a colour-split level)
__device__ __forceinline__ T restrict_at(const Level<T>& F, const Xfer<T>& X, const T* __restrict__ fine,
                                         int J0, int J1, int J2, bool cs = false) {
  T s = T(0);
  const int c0 = X.rc[0][J0], c1 = X.rc[1][J1], c2 = X.rc[2][J2];
  for (int a2 = 0; a2 < c2; ++a2) {
    const int f2 = X.ri[2][RMAX * J2 + a2];
    const T w2 = X.rw[2][RMAX * J2 + a2];
    for (int a1 = 0; a1 < c1; ++a1) {
      const int f1 = X.ri[1][RMAX * J1 + a1];
      const T w1 = X.rw[1][RMAX * J1 + a1];
      const long long row = (long long)F.n0 * (f1 + (long long)F.n1 * f2);
      for (int a0 = 0; a0 < c0; ++a0) {
        const T w0 = X.rw[0][RMAX * J0 + a0];
        const int f0 = X.ri[0][RMAX * J0 + a0];
        const long long idx = cs ? (long long)pix_of(1, F.n0, F.n1, F.n2, (unsigned)(row + f0), f0, f1, f2) : row + f0;
        s += w0 * w1 * w2 * fine[idx];
      }
    }
  }
  return s;
}

// sum_J P(i, J) (u_c - ubar_c)(J)
template <typename T>
__device__ __forceinline__ T prolong_at(const Level<T>& C, const Xfer<T>& X, int i0, int i1, int i2) {
  T s = T(0);
  const int c0 = X.pc[0][i0], c1 = X.pc[1][i1], c2 = X.pc[2][i2];
  for (int a2 = 0; a2 < c2; ++a2) {
    const int J2 = X.pj[2][2 * i2 + a2];
    const T w2 = X.pw[2][2 * i2 + a2];
    for (int a1 = 0; a1 < c1; ++a1) {
      const int J1 = X.pj[1][2 * i1 + a1];
      const T w1 = X.pw[1][2 * i1 + a1];
      const long long row = (long long)C.n0 * (J1 + (long long)C.n1 * J2);
      for (int a0 = 0; a0 < c0; ++a0) {
        const T w0 = X.pw[0][2 * i0 + a0];
        const long long J = row + X.pj[0][2 * i0 + a0];
        s += w0 * w1 * w2 * (C.u[J] - C.ubar[J]);
      }
    }
  }
  return s;
}

// ---------------------------------------------------------------------------
// max-norm reductions: |x| of finite or NaN values compares as its bit
// pattern (NaN sorts above +inf, so a NaN anywhere survives the max).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long nbits(double x) {
  return (unsigned long long)__double_as_longlong(fabs(x));
}
__device__ __forceinline__ unsigned long long nbits(float x) {
  return (unsigned long long)__float_as_uint(fabsf(x));
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// block-wide max of v; every thread gets the result (uses 33 words of smem)
__device__ __forceinline__ unsigned long long block_max(unsigned long long v, unsigned long long* sm) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    unsigned long long x = lane < nw ? sm[lane] : 0ull;
    x = warp_max(x);
    if (lane == 0) sm[32] = x;
  }
  __syncthreads();
  return sm[32];
}

}  // namespace rich
