// FP64 instantiations and the per-step preparation kernels.
#include "ddmath.cuh"
#include "kernels.cuh"

namespace rich {

using D = Dispatch<double, FORM_DIRECT>;
void sweep64(const Level<double>& L, const Phys<double>& P, int model, int color, cudaStream_t s) {
  D::sweep(L, P, model, color, s);
}
void residual64(const Level<double>& L, const Phys<double>& P, int model, unsigned long long* norm,
                cudaStream_t s) {
  D::residual(L, P, model, norm, s);
}
void tau64(const Level<double>& C, const Phys<double>& P, int model, cudaStream_t s) { D::tau(C, P, model, s); }
void restrict64(const Level<double>& F, const Level<double>& C, const Xfer<double>& X, const double* fa,
                const double* fb, double* ca, double* cb, cudaStream_t s) {
  D::restrict2(F, C, X, fa, fb, ca, cb, s);
}
void prolong64(const Level<double>& F, const Level<double>& C, const Xfer<double>& X, cudaStream_t s) {
  D::prolong(F, C, X, s);
}
void tail64(const Level<double>* dLs, const Xfer<double>* dXs, int l0, int nl, const Phys<double>& P, int model,
            int nu1, int nu2, int cmax, double crtol, int gamma, int gamma_levels, unsigned long long* stats,
            int ordering, cudaStream_t s) {
  D::tail(dLs, dXs, l0, nl, P, model, nu1, nu2, cmax, crtol, gamma, gamma_levels, stats, ordering, s);
}
void sweep_lex64(const Level<double>& L, const Phys<double>& P, int model, cudaStream_t s) { D::sweep_lex(L, P, model, s); }

// ---------------------------------------------------------------------------
// Lagged state and history (eq. fully-bdf1; BDF2 reading: a = 3/(2 tau),
// history (4 theta^n - theta^{n-1}) / (2 tau), psi* = 2 psi^n - psi^{n-1}):
//   Kc = K(psi*),  g = a*history + xi psi*,  u = psi^n (initial iterate).
// ---------------------------------------------------------------------------
template <int MODEL>
__global__ void __launch_bounds__(256) k_prep_lagged(long long n, const double* __restrict__ psin,
                                                     const double* __restrict__ psinm1, const double* __restrict__ Ks,
                                                     double Ks_s, const double* __restrict__ p1f,
                                                     const double* __restrict__ p2f, const uint8_t* __restrict__ mat,
                                                     Phys<double> P, int scheme, double hist_scale, double* Kc,
                                                     float* Kcf,
                                                     double* g, double* u, const double* thn_in,
                                                     const double* thm_in, double* thn_out, double* thm_out,
                                                     bool predict, const double* __restrict__ mf) {
  // thn_in / thm_in: theta(psi^n), theta(psi^{n-1}) kept from earlier FP64
  // evaluations (nullable: evaluate here, and keep them in *_out if given).
  // Kcf (nullable): an FP32 copy of Kc for the inner cycles of the mixed
  // mode; predict: the iterate starts at psi* instead of psi^n.
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double p1 = p1f ? p1f[i] : P.p1, p2 = p2f ? p2f[i] : P.p2;
    const double ks = Ks ? Ks[i] : Ks_s;
    const double pn = psin[i];
    with_law<MODEL>(P, mat_at<MODEL>(mat, i), [&](auto law, const Phys<double>& Q) {
      constexpr int ML = decltype(law)::value;
      // (the expression of the defect kernel's theta, so that a cache filled
      // here and one filled there hold the same bits for the same state)
      auto theta_at = [&](double x) {
        return (ML == VANGENUCHTEN && mf) ? theta_only_dm<ML>(x, p1, p2, mf[i], Q) : theta_only_d<ML>(x, p1, p2, Q);
      };
      double thn;
      if (thn_in) {
        thn = thn_in[i];
      } else {
        thn = theta_at(pn);
        if (thn_out) thn_out[i] = thn;
      }
      double ps, hist;
      if (scheme == 1) {
        ps = pn;
        hist = thn * hist_scale;
      } else {
        const double pm = psinm1[i];
        double thm;
        if (thm_in) {
          thm = thm_in[i];
        } else {
          thm = theta_at(pm);
          if (thm_out) thm_out[i] = thm;
        }
        ps = P.lag ? pn : 2.0 * pn - pm;
        hist = (4.0 * thn - thm) * hist_scale;
      }
      const double K = (ML == VANGENUCHTEN && mf) ? cond_dm<ML>(ps, p1, p2, mf[i], ks, Q)
                                                  : cond_d<ML>(ps, p1, p2, ks, Q);
      Kc[i] = K;
      if (Kcf) Kcf[i] = (float)K;
      g[i] = hist + P.xi * ps;
      u[i] = predict ? ps : pn;
      return 0;
    });
  }
}

// The same lagged state in float-float arithmetic (mixed mode): Kc = K(psi*)
// to FP64 (Kc) and FP32 (Kcf), g = history + xi psi* to FP64; theta(psi^n)
// and theta(psi^{n-1}) from the caches when given, else evaluated and kept.
template <int MODEL>
__global__ void __launch_bounds__(256) k_prep_lagged_dd(long long n, const double* __restrict__ psin,
                                                        const double* __restrict__ psinm1,
                                                        const double* __restrict__ Ks, dd Ks_s,
                                                        const double* __restrict__ p1f,
                                                        const double* __restrict__ p2f,
                                                        const uint8_t* __restrict__ mat, Phys<double> P, DDPhys Q,
                                                        int scheme, dd hist_scale, double* Kc, float* Kcf, double* g,
                                                        double* u, const double* thn_in, const double* thm_in,
                                                        double* thn_out, double* thm_out, bool predict) {
  // hist_scale: 1/tau (BDF1) or 1/(2 tau) (BDF2)
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const dd p1 = p1f ? dd_split(p1f[i]) : Q.p1, p2 = p2f ? dd_split(p2f[i]) : Q.p2;
    const double pnd = psin[i];
    const dd pn = dd_split(pnd);
    with_law_dd<MODEL>(P, Q, mat_at<MODEL>(mat, i), [&](auto law, const Phys<double>& Pc, const DDPhys& Qc) {
      constexpr int ML = decltype(law)::value;
      dd thn;
      if (thn_in) {
        thn = dd_split(thn_in[i]);
      } else {
        thn = theta_x<ML>(pn, p1, p2, Qc, Pc);
        if (thn_out) thn_out[i] = dd_join(thn);
      }
      dd ps, hist;
      if (scheme == 1) {
        ps = pn;
        hist = dd_mul(thn, hist_scale);
      } else {
        const dd pm = dd_split(psinm1[i]);
        dd thm;
        if (thm_in) {
          thm = dd_split(thm_in[i]);
        } else {
          thm = theta_x<ML>(pm, p1, p2, Qc, Pc);
          if (thm_out) thm_out[i] = dd_join(thm);
        }
        ps = Pc.lag ? pn : dd_sub(mk(2.0f * pn.hi, 2.0f * pn.lo), pm);
        hist = dd_mul(dd_sub(mk(4.0f * thn.hi, 4.0f * thn.lo), thm), hist_scale);
      }
      const dd K = cond_x<ML>(ps, p1, p2, Ks ? dd_split(Ks[i]) : Ks_s, Qc, Pc);
      Kc[i] = dd_join(K);
      Kcf[i] = dd_float(K);
      g[i] = dd_join(dd_add(hist, dd_mul(Q.xi, ps)));
      u[i] = predict ? dd_join(ps) : pnd;
      return 0;
    });
  }
}

// Gravity and boundary terms of g, and boundary face conductances:
//   gravity  -(M z)_i = (K_{i+e_z/2} - K_{i-e_z/2}) / h_z over interior faces,
//   Dirichlet (reading)  kb = (Kc_i + K(psi_b))/2,  g += 2 kb / h^2 (psi_b + z_b - z_i),
//   prescribed inflow q:  g += q / h,   free drainage:  g -= Kc_i / h_z.
template <int MODEL>
__global__ void __launch_bounds__(256) k_prep_rhs(Geom G, BcDev bc, const double* __restrict__ Ks, double Ks_s,
                                                  const double* __restrict__ p1f, const double* __restrict__ p2f,
                                                  const uint8_t* __restrict__ mat, Phys<double> P,
                                                  const double* __restrict__ Kc, double* g,
                                                  double* kb0, double* kb1, double* kb2, double* kb3, double* kb4,
                                                  double* kb5) {
  double* kb[6] = {kb0, kb1, kb2, kb3, kb4, kb5};
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const int v = G.dim - 1;
  const int nn[3] = {G.n0, G.n1, G.n2};
  const long long stride[3] = {1, G.n0, (long long)G.n0 * G.n1};
  const double ihv = 1.0 / G.h[v];    // (one FP64 division per thread, not two per cell)
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int ii[3];
    cell_coords(G.n0, G.n1, i, ii[0], ii[1], ii[2]);
    double gi = g[i];
    const double Ki = Kc[i];
    if (ii[v] + 1 < nn[v]) gi += 0.5 * (Ki + Kc[i + stride[v]]) * ihv;
    if (ii[v] > 0) gi -= 0.5 * (Ki + Kc[i - stride[v]]) * ihv;
    for (int ax = 0; ax < G.dim; ++ax) {
      for (int side = 0; side < 2; ++side) {
        if (ii[ax] != (side ? nn[ax] - 1 : 0)) continue;
        const int f = 2 * ax + side;
        long long fc;
        if (ax == 0) fc = ii[1] + (long long)G.n1 * ii[2];
        else if (ax == 1) fc = ii[0] + (long long)G.n0 * ii[2];
        else fc = ii[0] + (long long)G.n0 * ii[1];
        const double h = G.h[ax];
        const int kind = bc.kind[f];
        const bool dir = kind == 0 && (!bc.mask[f] || bc.mask[f][fc]);
        const double val = bc.vfield[f] ? bc.vfield[f][fc] : bc.value[f];
        if (dir) {
          const double p1 = p1f ? p1f[i] : P.p1, p2 = p2f ? p2f[i] : P.p2;
          const double ks = Ks ? Ks[i] : Ks_s;
          const double Kb = with_law<MODEL>(P, mat_at<MODEL>(mat, i), [&](auto law, const Phys<double>& Q) {
            return cond_d<decltype(law)::value>(val, p1, p2, ks, Q);
          });
          const double k = 0.5 * (Ki + Kb);
          kb[f][fc] = k;
          const double dz = (ax == v) ? (side ? 0.5 * h : -0.5 * h) : 0.0;
          gi += 2.0 * k / (h * h) * (val + dz);
        } else {
          kb[f][fc] = 0.0;
          if (kind == 2) gi += val / h;
          else if (kind == 3) gi -= Ki / h;
        }
      }
    }
    g[i] = gi;
  }
}

// The same gravity and boundary terms in float-float (mixed mode: no FP64
// arithmetic on the path; FP64 arrays split and joined with integer bit
// operations).  Per-axis constants split on the host: 0.5/h, 1/h, 2/h^2, h/2.
struct RhsConstDD {
  dd half_ih[3], ih[3], two_ih2[3], half_h[3];
};

template <int MODEL>
__global__ void __launch_bounds__(256) k_prep_rhs_dd(Geom G, BcDev bc, const double* __restrict__ Ks, dd Ks_s,
                                                     const double* __restrict__ p1f, const double* __restrict__ p2f,
                                                     const uint8_t* __restrict__ mat, Phys<double> P, DDPhys Q,
                                                     RhsConstDD H, const double* __restrict__ Kc, double* g,
                                                     double* kb0, double* kb1, double* kb2, double* kb3, double* kb4,
                                                     double* kb5) {
  double* kb[6] = {kb0, kb1, kb2, kb3, kb4, kb5};
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const int v = G.dim - 1;
  const int nn[3] = {G.n0, G.n1, G.n2};
  const long long stride[3] = {1, G.n0, (long long)G.n0 * G.n1};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int ii[3];
    cell_coords(G.n0, G.n1, i, ii[0], ii[1], ii[2]);
    dd gi = dd_split(g[i]);
    const dd Ki = dd_split(Kc[i]);
    if (ii[v] + 1 < nn[v]) gi = dd_add(gi, dd_mul(dd_add(Ki, dd_split(Kc[i + stride[v]])), H.half_ih[v]));
    if (ii[v] > 0) gi = dd_sub(gi, dd_mul(dd_add(Ki, dd_split(Kc[i - stride[v]])), H.half_ih[v]));
    for (int ax = 0; ax < G.dim; ++ax) {
      for (int side = 0; side < 2; ++side) {
        if (ii[ax] != (side ? nn[ax] - 1 : 0)) continue;
        const int f = 2 * ax + side;
        long long fc;
        if (ax == 0) fc = ii[1] + (long long)G.n1 * ii[2];
        else if (ax == 1) fc = ii[0] + (long long)G.n0 * ii[2];
        else fc = ii[0] + (long long)G.n0 * ii[1];
        const int kind = bc.kind[f];
        const bool dir = kind == 0 && (!bc.mask[f] || bc.mask[f][fc]);
        const dd val = dd_split(bc.vfield[f] ? bc.vfield[f][fc] : bc.value[f]);
        if (dir) {
          const dd p1 = p1f ? dd_split(p1f[i]) : Q.p1, p2 = p2f ? dd_split(p2f[i]) : Q.p2;
          const dd ks = Ks ? dd_split(Ks[i]) : Ks_s;
          const dd Kb = with_law_dd<MODEL>(P, Q, mat_at<MODEL>(mat, i),
                                           [&](auto law, const Phys<double>& Pc, const DDPhys& Qc) {
                                             return cond_x<decltype(law)::value>(val, p1, p2, ks, Qc, Pc);
                                           });
          const dd ksum = dd_add(Ki, Kb);
          const dd k = mk(0.5f * ksum.hi, 0.5f * ksum.lo);
          kb[f][fc] = dd_join(k);
          dd head = val;
          if (ax == v) head = side ? dd_add(val, H.half_h[ax]) : dd_sub(val, H.half_h[ax]);
          gi = dd_add(gi, dd_mul(dd_mul(k, H.two_ih2[ax]), head));
        } else {
          kb[f][fc] = 0.0;
          if (kind == 2) gi = dd_add(gi, dd_mul(val, H.ih[ax]));
          else if (kind == 3) gi = dd_sub(gi, dd_mul(Ki, H.ih[ax]));
        }
      }
    }
    g[i] = dd_join(gi);
  }
}

// restriction of a boundary-face array over the face's two in-plane axes
template <typename T>
__global__ void __launch_bounds__(256) k_restrict_face(Geom F, Geom C, Xfer<T> X, int ax, const T* fine, T* coarse) {
  int oa[2], k = 0;
  for (int a = 0; a < 3; ++a)
    if (a != ax) oa[k++] = a;
  const int nF[3] = {F.n0, F.n1, F.n2}, nC[3] = {C.n0, C.n1, C.n2};
  const long long nc = (long long)nC[oa[0]] * nC[oa[1]];
  for (long long J = blockIdx.x * (long long)blockDim.x + threadIdx.x; J < nc; J += (long long)gridDim.x * blockDim.x) {
    const int J0 = (int)(J % nC[oa[0]]), J1 = (int)(J / nC[oa[0]]);
    const int c0 = X.rc[oa[0]][J0], c1 = X.rc[oa[1]][J1];
    T s = T(0);
    for (int a1 = 0; a1 < c1; ++a1)
      for (int a0 = 0; a0 < c0; ++a0)
        s += X.rw[oa[0]][RMAX * J0 + a0] * X.rw[oa[1]][RMAX * J1 + a1] *
             fine[X.ri[oa[0]][RMAX * J0 + a0] + (long long)nF[oa[0]] * X.ri[oa[1]][RMAX * J1 + a1]];
    coarse[J] = s;
  }
}

// Sink coefficient (reading): Tp exp(-depth/decay) normalised over the root
// zone [0, root_depth], depth measured down from the top face.
__global__ void __launch_bounds__(256) k_sink_coef(Geom G, double Tp, double D, double lam, double* smax) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const int v = G.dim - 1;
  const double Z = lam * (1.0 - exp(-D / lam));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int ii[3];
    cell_coords(G.n0, G.n1, i, ii[0], ii[1], ii[2]);
    // centre depth below the top face as one product and one quotient, so the
    // root-zone edge is decided identically whatever the compiler fuses
    const int nv = v == 0 ? G.n0 : (v == 1 ? G.n1 : G.n2);
    const double depth = G.Lv * (double)(2 * (nv - 1 - ii[v]) + 1) / (double)(2 * nv);
    smax[i] = depth <= D ? Tp * exp(-depth / lam) / Z : 0.0;
  }
}

__global__ void __launch_bounds__(256) k_to_float(const double* src, float* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// Defect of the mixed mode's outer loop, d = g - N(u) (eq. Nh-def), in
// float-float arithmetic (no FP64 instruction on the path: the FP64 arrays
// are split with integer operations); hands the FP32 inner problem its right
// side d, its frozen state psi0 = u and a zero initial correction, and
// accumulates ||d||_inf (as float bits).  The interior fluxes are taken in
// difference form m_f (u_i - u_j), so nothing cancels.  theta(u) comes from
// th_in when given (u = psi^n), else it is evaluated and kept in th_out
// (nullable) for the next step's history.
template <int MODEL>
__global__ void __launch_bounds__(128) k_outer_residual_dd(Level<double> L, Phys<double> P, DDPhys Q, float* r32,
                                                           float* psi0f, float* delta, unsigned long long* norm,
                                                           const double* __restrict__ th_in, double* th_out, int cs) {
  __shared__ unsigned long long sm[33];
  unsigned long long mx = 0;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int i1 = blockIdx.y, i2 = blockIdx.z;
  if (i0 < L.n0) {
    const long long i = i0 + (long long)L.n0 * (i1 + (long long)L.n1 * i2);
    const double* __restrict__ u = L.u;
    const double* __restrict__ K = L.Kc;
    const dd ui = dd_split(u[i]);
    const dd Ki = dd_split(K[i]);
    dd flux = mk(0.0f), db = mk(0.0f);
    const int nn[3] = {L.n0, L.n1, L.n2};
    const int ii[3] = {i0, i1, i2};
    const long long st[3] = {1, L.n0, (long long)L.n0 * L.n1};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= L.dim) break;
      const dd s = dd_split(L.ih2[a]), hs = mk(0.5f * s.hi, 0.5f * s.lo), s2 = mk(2.0f * s.hi, 2.0f * s.lo);
      long long fc;
      if (a == 0) fc = i1 + (long long)L.n1 * i2;
      else if (a == 1) fc = i0 + (long long)L.n0 * i2;
      else fc = i0 + (long long)L.n0 * i1;
      if (ii[a] > 0) {
        const long long j = i - st[a];
        flux = dd_add(flux, dd_mul(dd_mul(dd_add(Ki, dd_split(K[j])), hs), dd_sub(ui, dd_split(u[j]))));
      } else {
        db = dd_add(db, dd_mul(dd_split(L.kb[2 * a][fc]), s2));
      }
      if (ii[a] < nn[a] - 1) {
        const long long j = i + st[a];
        flux = dd_add(flux, dd_mul(dd_mul(dd_add(Ki, dd_split(K[j])), hs), dd_sub(ui, dd_split(u[j]))));
      } else {
        db = dd_add(db, dd_mul(dd_split(L.kb[2 * a + 1][fc]), s2));
      }
    }
    dd th;
    if (th_in) {
      th = dd_split(th_in[i]);
    } else {
      const dd p1 = L.p1 ? dd_split(L.p1[i]) : Q.p1, p2 = L.p2 ? dd_split(L.p2[i]) : Q.p2;
      th = with_law_dd<MODEL>(P, Q, mat_of<MODEL>(L, i), [&](auto law, const Phys<double>& Pc, const DDPhys& Qc) {
        return theta_x<decltype(law)::value>(ui, p1, p2, Qc, Pc);
      });
      if (th_out) th_out[i] = dd_join(th);
    }
    const dd S = L.smax ? sink_x(ui, dd_split(L.smax[i]), Q) : mk(0.0f);
    // N = a theta + S + xi u + sum_f m_f (u_i - u_j) + (sum of Dirichlet diagonals) u
    dd N = dd_add(dd_mul(Q.a, th), S);
    N = dd_add(N, dd_mul(dd_add(Q.xi, db), ui));
    N = dd_add(N, flux);
    const float di = dd_float(dd_sub(dd_split(L.g[i]), N));
    const unsigned q = pix_of(cs, L.n0, L.n1, L.n2, (unsigned)i, i0, i1, i2);
    r32[q] = di;
    psi0f[q] = dd_float(ui);
    delta[i] = 0.0f;
    mx = nbits(di);
  }
  mx = block_max(mx, sm);
  if (threadIdx.x == 0) atomicMax(norm, mx);
}

// The same defect in FP64 (the FP64-outer mixed mode's accepting defect and
// stop test): d = g - N(u) (eq. Nh-def) with the interior fluxes in
// difference form m_f (u_i - u_j), as k_outer_residual_dd takes them -- the
// form m_ii u_i - sum_j m_ij u_j of the grid residual would cancel the large
// diagonal of a fine, conductive level (terms ~1e5 in theta units) down to
// rounding above a tight tolerance.  theta in FP64 from th_in when given
// (u = psi^n), else evaluated and kept in th_out (nullable) for the next
// step's history.  Hands the FP32 inner problem r32, psi0 and a zero
// correction like k_outer_residual_dd; ||d||_inf accumulates as FP64 bits.
template <int MODEL>
__global__ void __launch_bounds__(256) k_outer_residual64(Level<double> L, Phys<double> P, float* r32, float* psi0f,
                                                          float* delta, unsigned long long* norm,
                                                          const double* __restrict__ th_in, double* th_out, int cs,
                                                          const double* __restrict__ mf) {
  __shared__ unsigned long long sm[33];
  unsigned long long mx = 0;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int i1 = blockIdx.y, i2 = blockIdx.z;
  if (i0 < L.n0) {
    const long long i = (unsigned)(i0 + L.n0 * (i1 + L.n1 * i2));
    const double* __restrict__ u = L.u;
    const double* __restrict__ K = L.Kc;
    const double ui = u[i], Ki = K[i];
    double flux = 0.0, db = 0.0;
    const int nn[3] = {L.n0, L.n1, L.n2};
    const int ii[3] = {i0, i1, i2};
    const long long st[3] = {1, L.n0, (long long)L.n0 * L.n1};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= L.dim) break;
      const double s = L.ih2[a], hs = 0.5 * s;
      long long fc;
      if (a == 0) fc = i1 + (long long)L.n1 * i2;
      else if (a == 1) fc = i0 + (long long)L.n0 * i2;
      else fc = i0 + (long long)L.n0 * i1;
      if (ii[a] > 0) flux += (Ki + K[i - st[a]]) * hs * (ui - u[i - st[a]]);
      else db += 2.0 * L.kb[2 * a][fc] * s;
      if (ii[a] < nn[a] - 1) flux += (Ki + K[i + st[a]]) * hs * (ui - u[i + st[a]]);
      else db += 2.0 * L.kb[2 * a + 1][fc] * s;
    }
    double th;
    if (th_in) {
      th = th_in[i];
    } else {
      const double p1 = L.p1 ? L.p1[i] : P.p1, p2 = L.p2 ? L.p2[i] : P.p2;
      th = with_law<MODEL>(P, mat_of<MODEL>(L, i), [&](auto law, const Phys<double>& Q) {
        constexpr int ML = decltype(law)::value;
        return (ML == VANGENUCHTEN && mf) ? theta_only_dm<ML>(ui, p1, p2, mf[i], Q)
                                          : theta_only_d<ML>(ui, p1, p2, Q);
      });
      if (th_out) th_out[i] = th;
    }
    double S, dS;
    sink_direct(ui, L.smax ? L.smax[i] : 0.0, P, S, dS);
    const double di = L.g[i] - ((P.a * th + S) + (P.xi + db) * ui + flux);
    const unsigned q = pix_of(cs, L.n0, L.n1, L.n2, (unsigned)i, i0, i1, i2);
    r32[q] = (float)di;
    psi0f[q] = (float)ui;
    delta[i] = 0.0f;
    mx = nbits(di);
  }
  mx = block_max(mx, sm);
  if (threadIdx.x == 0) atomicMax(norm, mx);
}

__global__ void __launch_bounds__(256) k_apply_delta(double* u, const float* delta, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    u[i] += (double)delta[i];
}

void prep_lagged(const Geom& G, const double* psin, const double* psinm1, const double* Ks, double Ks_s,
                 const double* p1, const double* p2, const uint8_t* mat, const Phys<double>& P, int model, int scheme,
                 double dt, double* Kc, float* Kcf, double* g, double* u, const double* thn_in,
                 const double* thm_in, double* thn_out, double* thm_out, bool predict, cudaStream_t s,
                 const double* vgm) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const int b = grid_for(n);
  predict = predict && scheme == 2;
  by_model(model, [&](auto m) {
    // (the history's 1/tau or 1/(2 tau) as one factor, as in the water balance)
    const double hs = scheme == 1 ? 1.0 / dt : 1.0 / (2.0 * dt);
    k_prep_lagged<decltype(m)::value><<<b, 256, 0, s>>>(n, psin, psinm1, Ks, Ks_s, p1, p2, mat, P, scheme, hs, Kc,
                                                        Kcf, g, u, thn_in, thm_in, thn_out, thm_out, predict,
                                                        decltype(m)::value == VANGENUCHTEN ? vgm : nullptr);
  });
}

void prep_lagged_dd(const Geom& G, const double* psin, const double* psinm1, const double* Ks, double Ks_s,
                    const double* p1, const double* p2, const uint8_t* mat, const Phys<double>& P, const DDPhys& Q,
                    int model, int scheme, double dt, double* Kc, float* Kcf, double* g, double* u,
                    const double* thn_in, const double* thm_in, double* thn_out, double* thm_out, bool predict,
                    cudaStream_t s) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const int b = grid_for(n);
  const dd ks = host_split(Ks_s), hs = host_split(scheme == 1 ? 1.0 / dt : 1.0 / (2.0 * dt));
  predict = predict && scheme == 2;
  by_model(model, [&](auto m) {
    k_prep_lagged_dd<decltype(m)::value><<<b, 256, 0, s>>>(n, psin, psinm1, Ks, ks, p1, p2, mat, P, Q, scheme, hs, Kc,
                                                           Kcf, g, u, thn_in, thm_in, thn_out, thm_out, predict);
  });
}

void prep_rhs(const Geom& G, const BcDev& bc, const double* Ks, double Ks_s, const double* p1, const double* p2,
              const uint8_t* mat, const Phys<double>& P, int model, const double* Kc, double* g, double* const kb[6],
              cudaStream_t s) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const int b = grid_for(n);
  by_model(model, [&](auto m) {
    k_prep_rhs<decltype(m)::value><<<b, 256, 0, s>>>(G, bc, Ks, Ks_s, p1, p2, mat, P, Kc, g, kb[0], kb[1], kb[2], kb[3],
                                                     kb[4], kb[5]);
  });
}

void prep_rhs_dd(const Geom& G, const BcDev& bc, const double* Ks, double Ks_s, const double* p1, const double* p2,
                 const uint8_t* mat, const Phys<double>& P, const DDPhys& Q, int model, const double* Kc, double* g,
                 double* const kb[6], cudaStream_t s) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const int b = grid_for(n);
  RhsConstDD H;
  for (int a = 0; a < 3; ++a) {
    const double h = G.h[a];
    H.half_ih[a] = host_split(0.5 / h);
    H.ih[a] = host_split(1.0 / h);
    H.two_ih2[a] = host_split(2.0 / (h * h));
    H.half_h[a] = host_split(0.5 * h);
  }
  const dd ks = host_split(Ks_s);
  by_model(model, [&](auto m) {
    k_prep_rhs_dd<decltype(m)::value><<<b, 256, 0, s>>>(G, bc, Ks, ks, p1, p2, mat, P, Q, H, Kc, g, kb[0], kb[1], kb[2],
                                                        kb[3], kb[4], kb[5]);
  });
}

void restrict_face64(const Geom& F, const Geom& C, const Xfer<double>& X, int axis, const double* fine,
                     double* coarse, cudaStream_t s) {
  const int nC[3] = {C.n0, C.n1, C.n2};
  long long nc = 1;
  for (int a = 0; a < 3; ++a)
    if (a != axis) nc *= nC[a];
  k_restrict_face<double><<<grid_for(nc), 256, 0, s>>>(F, C, X, axis, fine, coarse);
}

void restrict_face32(const Geom& F, const Geom& C, const Xfer<float>& X, int axis, const float* fine, float* coarse,
                     cudaStream_t s) {
  const int nC[3] = {C.n0, C.n1, C.n2};
  long long nc = 1;
  for (int a = 0; a < 3; ++a)
    if (a != axis) nc *= nC[a];
  k_restrict_face<float><<<grid_for(nc), 256, 0, s>>>(F, C, X, axis, fine, coarse);
}

void sink_coef(const Geom& G, double Tp, double depth, double decay, double* smax, cudaStream_t s) {
  k_sink_coef<<<grid_for((long long)G.n0 * G.n1 * G.n2), 256, 0, s>>>(G, Tp, depth, decay, smax);
}

void to_float(const double* src, float* dst, long long n, cudaStream_t s) {
  k_to_float<<<grid_for(n), 256, 0, s>>>(src, dst, n);
}

void outer_residual_dd(const Level<double>& L, const Phys<double>& P, const DDPhys& Q, int model, float* r32,
                       float* psi0f, float* delta, unsigned long long* norm, const double* th_in, double* th_out,
                       int cs, cudaStream_t s) {
  const Launch3 g = launch3(L.n0, L.n1, L.n2);
  by_model(model, [&](auto m) {
    k_outer_residual_dd<decltype(m)::value><<<g.grid, g.block, 0, s>>>(L, P, Q, r32, psi0f, delta, norm, th_in,
                                                                       th_out, cs);
  });
}

void outer_residual64(const Level<double>& L, const Phys<double>& P, int model, float* r32, float* psi0f,
                      float* delta, unsigned long long* norm, const double* th_in, double* th_out, int cs,
                      cudaStream_t s, const double* vgm) {
  const Launch3 g = launch3(L.n0, L.n1, L.n2);
  by_model(model, [&](auto m) {
    k_outer_residual64<decltype(m)::value><<<g.grid, g.block, 0, s>>>(L, P, r32, psi0f, delta, norm, th_in, th_out,
                                                                      cs, decltype(m)::value == VANGENUCHTEN ? vgm
                                                                                                           : nullptr);
  });
}

// m = 1 - 1/n of a van Genuchten n field (vg_m, the laws' own expression)
__global__ void __launch_bounds__(256) k_vg_m(const double* __restrict__ n, double* m, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    m[i] = vg_m(n[i]);
}

void vg_m_field(const double* n, double* m, long long count, cudaStream_t s) {
  k_vg_m<<<grid_for(count), 256, 0, s>>>(n, m, count);
}

__global__ void __launch_bounds__(256) k_to_float_level(const double* __restrict__ src, float* dst, int n0, int n1,
                                                        int n2, int cs) {
  const long long n = (long long)n0 * n1 * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int i0, i1, i2;
    cell_coords(n0, n1, i, i0, i1, i2);
    dst[pix_of(cs, n0, n1, n2, (unsigned)i, i0, i1, i2)] = (float)src[i];
  }
}

__global__ void __launch_bounds__(256) k_cs_to_natural(const float* __restrict__ src, float* dst, int n0, int n1,
                                                       int n2) {
  const long long n = (long long)n0 * n1 * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int i0, i1, i2;
    cell_coords(n0, n1, i, i0, i1, i2);
    dst[i] = src[pix_of(1, n0, n1, n2, (unsigned)i, i0, i1, i2)];
  }
}

void to_float_level(const double* src, float* dst, int n0, int n1, int n2, int cs, cudaStream_t s) {
  k_to_float_level<<<grid_for((long long)n0 * n1 * n2), 256, 0, s>>>(src, dst, n0, n1, n2, cs);
}

void cs_to_natural(const float* src, float* dst, int n0, int n1, int n2, cudaStream_t s) {
  k_cs_to_natural<<<grid_for((long long)n0 * n1 * n2), 256, 0, s>>>(src, dst, n0, n1, n2);
}

template <int MODEL, bool DD>
__global__ void __launch_bounds__(256) k_soil_eval(long long n, const double* __restrict__ psi,
                                                   const double* __restrict__ Ks, double Ks_s,
                                                   const double* __restrict__ p1f, const double* __restrict__ p2f,
                                                   const uint8_t* __restrict__ mat, Phys<double> P, DDPhys Q,
                                                   double* theta, double* K) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double p1 = p1f ? p1f[i] : P.p1, p2 = p2f ? p2f[i] : P.p2, x = psi[i];
    const double ks = Ks ? Ks[i] : Ks_s;
    with_law_dd<MODEL>(P, Q, mat_at<MODEL>(mat, i), [&](auto law, const Phys<double>& Pc, const DDPhys& Qc) {
      constexpr int ML = decltype(law)::value;
      if (theta) theta[i] = DD ? theta_dd<ML>(x, p1, p2, Qc, Pc) : theta_only_d<ML>(x, p1, p2, Pc);
      if (K) K[i] = DD ? cond_dd<ML>(x, p1, p2, ks, Qc, Pc) : cond_d<ML>(x, p1, p2, ks, Pc);
      return 0;
    });
  }
}

template <bool DD>
static void soil_eval_t(long long n, const double* psi, const double* Ks, double Ks_s, const double* p1,
                        const double* p2, const uint8_t* mat, const Phys<double>& P, const DDPhys& Q, int model,
                        double* theta, double* K, cudaStream_t s) {
  const int b = grid_for(n);
  by_model(model, [&](auto m) {
    k_soil_eval<decltype(m)::value, DD><<<b, 256, 0, s>>>(n, psi, Ks, Ks_s, p1, p2, mat, P, Q, theta, K);
  });
}

void soil_eval(long long n, const double* psi, const double* Ks, double Ks_s, const double* p1, const double* p2,
               const uint8_t* mat, const Phys<double>& P, const DDPhys& Q, int model, bool dd, double* theta,
               double* K, cudaStream_t s) {
  if (dd) soil_eval_t<true>(n, psi, Ks, Ks_s, p1, p2, mat, P, Q, model, theta, K, s);
  else soil_eval_t<false>(n, psi, Ks, Ks_s, p1, p2, mat, P, Q, model, theta, K, s);
}

// ---------------------------------------------------------------------------
// Water balance of a step (float-float, per block partial sums).  Per cell,
//   V (a theta(psi) - hist + S(psi) + xi (psi - psi*)) - (boundary inflow of the cell),
// whose sum is -V sum_i r_i (r = g - N(psi)): interior fluxes telescope and
// the gravity and boundary terms of g are the boundary inflow.  Also the
// minimum over cells of a theta'(psi) + S'(psi) + xi (FP32), for the error
// bound ||psi - psi_exact|| <= ||N(psi) - g|| / min(...).
// ---------------------------------------------------------------------------
__device__ __forceinline__ dd warp_sum_dd(dd v) {
  for (int o = 16; o > 0; o >>= 1) {
    dd w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = dd_add(v, w);
  }
  return v;
}

template <int MODEL>
__global__ void __launch_bounds__(256) k_mass_balance(Level<double> L, Geom G, BcDev bc, Phys<double> P, DDPhys Q,
                                                      Phys<float> Pf, const double* __restrict__ psin,
                                                      const double* __restrict__ psinm1, int scheme, dd hist_scale,
                                                      const double* th_new, const double* th_n, const double* th_nm1,
                                                      double* part, unsigned* dmin_bits) {
  __shared__ float sh[2][32];
  dd acc = mk(0.0f);
  float dmin = __int_as_float(0x7f800000);
  const int v = G.dim - 1;
  const int nn[3] = {G.n0, G.n1, G.n2};
  double Vd = 1.0;
  for (int a = 0; a < G.dim; ++a) Vd *= G.h[a];
  const dd V = dd_split(Vd);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.ncell;
       i += (long long)gridDim.x * blockDim.x) {
    int ii[3];
    cell_coords(G.n0, G.n1, i, ii[0], ii[1], ii[2]);
    const dd p1 = L.p1 ? dd_split(L.p1[i]) : Q.p1, p2 = L.p2 ? dd_split(L.p2[i]) : Q.p2;
    const dd psi = dd_split(L.u[i]), pn = dd_split(psin[i]);
    const unsigned mi = mat_of<MODEL>(L, i);
    dd th1, thn, hist, ps;
    with_law_dd<MODEL>(P, Q, mi, [&](auto law, const Phys<double>& Pc, const DDPhys& Qc) {
      constexpr int ML = decltype(law)::value;
      th1 = th_new ? dd_split(th_new[i]) : theta_x<ML>(psi, p1, p2, Qc, Pc);
      thn = th_n ? dd_split(th_n[i]) : theta_x<ML>(pn, p1, p2, Qc, Pc);
      if (scheme == 1) {
        hist = dd_mul(thn, hist_scale);
        ps = pn;
      } else {
        const dd pm = dd_split(psinm1[i]);
        const dd thm = th_nm1 ? dd_split(th_nm1[i]) : theta_x<ML>(pm, p1, p2, Qc, Pc);
        hist = dd_mul(dd_sub(mk(4.0f * thn.hi, 4.0f * thn.lo), thm), hist_scale);
        ps = Pc.lag ? pn : dd_sub(mk(2.0f * pn.hi, 2.0f * pn.lo), pm);
      }
      return 0;
    });
    const dd smax = L.smax ? dd_split(L.smax[i]) : mk(0.0f);
    dd cell = dd_sub(dd_mul(Q.a, th1), hist);
    cell = dd_add(cell, sink_x(psi, smax, Q));
    cell = dd_add(cell, dd_mul(Q.xi, dd_sub(psi, ps)));
    cell = dd_mul(V, cell);
    // inflow through this cell's boundary faces (face area A = V / h)
    for (int ax = 0; ax < G.dim; ++ax)
      for (int side = 0; side < 2; ++side) {
        if (ii[ax] != (side ? nn[ax] - 1 : 0)) continue;
        const int f = 2 * ax + side;
        long long fc;
        if (ax == 0) fc = ii[1] + (long long)G.n1 * ii[2];
        else if (ax == 1) fc = ii[0] + (long long)G.n0 * ii[2];
        else fc = ii[0] + (long long)G.n0 * ii[1];
        const dd A = dd_split(Vd / G.h[ax]);
        const int kind = bc.kind[f];
        const bool dir = kind == 0 && (!bc.mask[f] || bc.mask[f][fc]);
        dd qin = mk(0.0f);
        if (dir) {
          const double zi = (ii[v] + 0.5) * G.h[v];
          const double zb = (ax == v) ? (side ? G.Lv : 0.0) : zi;
          const double val = bc.vfield[f] ? bc.vfield[f][fc] : bc.value[f];
          const dd head = dd_sub(dd_add(dd_split(val), dd_split(zb)), dd_add(psi, dd_split(zi)));
          qin = dd_mul(dd_mul(A, dd_split(L.kb[f][fc])), dd_mul(head, dd_split(2.0 / G.h[ax])));
        } else if (kind == 2) {
          qin = dd_mul(A, dd_split(bc.vfield[f] ? bc.vfield[f][fc] : bc.value[f]));
        } else if (kind == 3) {
          qin = dd_neg(dd_mul(A, dd_split(L.Kc[i])));
        }
        cell = dd_sub(cell, qin);
      }
    acc = dd_add(acc, cell);
    // a theta' + S' + xi at psi (FP32 increment laws with a zero increment)
    const float psif = dd_float(psi), p1f = dd_float(p1), p2f = dd_float(p2);
    float Dth, dth;
    with_law<MODEL>(Pf, mi, [&](auto law, const Phys<float>& Qf) {
      constexpr int ML = decltype(law)::value;
      dincr<ML>(dbase<ML>(psif, p1f, p2f), 0.0f, p1f, p2f, Qf, Dth, dth);
      return 0;
    });
    const float smf = dd_float(smax);
    float sa = 0.0f, sda = 0.0f;
    if (Pf.sink && smf > 0.0f) feddes(psif, Pf, sa, sda);
    dmin = fminf(dmin, Pf.a * dth + sda * smf + Pf.xi);
  }
  acc = warp_sum_dd(acc);
  for (int o = 16; o > 0; o >>= 1) dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh[0][wid] = acc.hi; sh[1][wid] = acc.lo; }
  __shared__ float smin[32];
  if (lane == 0) smin[wid] = dmin;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    dd x = lane < nw ? mk(sh[0][lane], sh[1][lane]) : mk(0.0f);
    float m = lane < nw ? smin[lane] : __int_as_float(0x7f800000);
    x = warp_sum_dd(x);
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      part[blockIdx.x] = dd_join(x);
      atomicMin(dmin_bits, __float_as_uint(fmaxf(m, 0.0f)));
    }
  }
}

// The same water balance in FP64 (FP64 mode and the FP64-outer mixed mode):
// theta from the FP64 caches where given, else FP64 laws; FP64 sums.  The
// error bound's minimum stays the FP32 expression of k_mass_balance.
template <int MODEL>
__global__ void __launch_bounds__(256) k_mass_balance64(Level<double> L, Geom G, BcDev bc, Phys<double> P,
                                                        Phys<float> Pf, const double* __restrict__ psin,
                                                        const double* __restrict__ psinm1, int scheme,
                                                        double hist_scale, const double* th_new, const double* th_n,
                                                        const double* th_nm1, double* part, unsigned* dmin_bits) {
  __shared__ double sh[32];
  __shared__ float smin[32];
  double acc = 0.0;
  float dmin = __int_as_float(0x7f800000);
  const int v = G.dim - 1;
  const int nn[3] = {G.n0, G.n1, G.n2};
  double V = 1.0;
  for (int a = 0; a < G.dim; ++a) V *= G.h[a];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.ncell;
       i += (long long)gridDim.x * blockDim.x) {
    int ii[3];
    cell_coords(G.n0, G.n1, i, ii[0], ii[1], ii[2]);
    const double p1 = L.p1 ? L.p1[i] : P.p1, p2 = L.p2 ? L.p2[i] : P.p2;
    const double psi = L.u[i], pn = psin[i];
    const unsigned mi = mat_of<MODEL>(L, i);
    double th1, hist, ps;
    with_law<MODEL>(P, mi, [&](auto law, const Phys<double>& Q) {
      constexpr int ML = decltype(law)::value;
      th1 = th_new ? th_new[i] : theta_only_d<ML>(psi, p1, p2, Q);
      const double thn = th_n ? th_n[i] : theta_only_d<ML>(pn, p1, p2, Q);
      if (scheme == 1) {
        hist = thn * hist_scale;
        ps = pn;
      } else {
        const double pm = psinm1[i];
        const double thm = th_nm1 ? th_nm1[i] : theta_only_d<ML>(pm, p1, p2, Q);
        hist = (4.0 * thn - thm) * hist_scale;
        ps = Q.lag ? pn : 2.0 * pn - pm;
      }
      return 0;
    });
    const double smax = L.smax ? L.smax[i] : 0.0;
    double S, dS;
    sink_direct(psi, smax, P, S, dS);
    double cell = (P.a * th1 - hist) + S + P.xi * (psi - ps);
    cell *= V;
    // inflow through this cell's boundary faces (face area A = V / h)
    for (int ax = 0; ax < G.dim; ++ax)
      for (int side = 0; side < 2; ++side) {
        if (ii[ax] != (side ? nn[ax] - 1 : 0)) continue;
        const int f = 2 * ax + side;
        long long fc;
        if (ax == 0) fc = ii[1] + (long long)G.n1 * ii[2];
        else if (ax == 1) fc = ii[0] + (long long)G.n0 * ii[2];
        else fc = ii[0] + (long long)G.n0 * ii[1];
        const double A = V / G.h[ax];
        const int kind = bc.kind[f];
        const bool dir = kind == 0 && (!bc.mask[f] || bc.mask[f][fc]);
        double qin = 0.0;
        if (dir) {
          const double zi = (ii[v] + 0.5) * G.h[v];
          const double zb = (ax == v) ? (side ? G.Lv : 0.0) : zi;
          const double val = bc.vfield[f] ? bc.vfield[f][fc] : bc.value[f];
          const double head = (val + zb) - (psi + zi);
          qin = A * L.kb[f][fc] * (head * (2.0 / G.h[ax]));
        } else if (kind == 2) {
          qin = A * (bc.vfield[f] ? bc.vfield[f][fc] : bc.value[f]);
        } else if (kind == 3) {
          qin = -A * L.Kc[i];
        }
        cell -= qin;
      }
    acc += cell;
    // a theta' + S' + xi at psi (FP32 increment laws with a zero increment)
    const float psif = (float)psi, p1f = (float)p1, p2f = (float)p2;
    float Dth, dth;
    with_law<MODEL>(Pf, mi, [&](auto law, const Phys<float>& Qf) {
      constexpr int ML = decltype(law)::value;
      dincr<ML>(dbase<ML>(psif, p1f, p2f), 0.0f, p1f, p2f, Qf, Dth, dth);
      return 0;
    });
    const float smf = (float)smax;
    float sa = 0.0f, sda = 0.0f;
    if (Pf.sink && smf > 0.0f) feddes(psif, Pf, sa, sda);
    dmin = fminf(dmin, Pf.a * dth + sda * smf + Pf.xi);
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh[wid] = acc; smin[wid] = dmin; }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double x = lane < nw ? sh[lane] : 0.0;
    float m = lane < nw ? smin[lane] : __int_as_float(0x7f800000);
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
      part[blockIdx.x] = x;
      atomicMin(dmin_bits, __float_as_uint(fmaxf(m, 0.0f)));
    }
  }
}

int mass_balance(const Level<double>& L, const Geom& G, const BcDev& bc, const Phys<double>& P, const Phys<float>& Pf,
                 int model, const double* psin, const double* psinm1, int scheme, double dt, const double* th_new,
                 const double* th_n, const double* th_nm1, double* part, unsigned* dmin_bits, bool fp64,
                 cudaStream_t s) {
  const int b = grid_for(L.ncell);
  if (fp64) {
    const double hs = scheme == 1 ? 1.0 / dt : 1.0 / (2.0 * dt);
    by_model(model, [&](auto m) {
      k_mass_balance64<decltype(m)::value><<<b, 256, 0, s>>>(L, G, bc, P, Pf, psin, psinm1, scheme, hs, th_new, th_n,
                                                             th_nm1, part, dmin_bits);
    });
    return b;
  }
  const DDPhys Q = make_ddphys(P);
  const dd hs = host_split(scheme == 1 ? 1.0 / dt : 1.0 / (2.0 * dt));
  by_model(model, [&](auto m) {
    k_mass_balance<decltype(m)::value><<<b, 256, 0, s>>>(L, G, bc, P, Q, Pf, psin, psinm1, scheme, hs, th_new, th_n,
                                                         th_nm1, part, dmin_bits);
  });
  return b;
}

// *flags |= 1 if any of x[0..n) is not finite (the exponent field all ones:
// integer test, so no FP64 instruction); with ref, *flags |= changed_bit if
// any x[i] differs from ref[i] in its bits (-0 and +0 differ)
__global__ void __launch_bounds__(256) k_screen(const double* __restrict__ x, const double* __restrict__ ref,
                                                long long n, unsigned changed_bit, unsigned* flags) {
  bool nf = false, ch = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x[i]);
    nf |= ((b >> 52) & 0x7ffull) == 0x7ffull;
    if (ref) ch |= b != (unsigned long long)__double_as_longlong(ref[i]);
  }
  const unsigned v = __reduce_or_sync(0xffffffffu, (nf ? 1u : 0u) | (ch ? changed_bit : 0u));
  if (v && (threadIdx.x & 31) == 0) atomicOr(flags, v);
}

void screen_state(const double* x, const double* ref, long long n, unsigned changed_bit, unsigned* flags,
                  cudaStream_t s) {
  k_screen<<<grid_for(n), 256, 0, s>>>(x, ref, n, changed_bit, flags);
}

void apply_delta(double* u, const float* delta, long long n, cudaStream_t s) {
  k_apply_delta<<<grid_for(n), 256, 0, s>>>(u, delta, n);
}

// The FP64 elementary functions of the laws (fn 0 exp, 1 expm1, 2 log,
// 3 log1p) and, for comparison, CUDA's (fn 4..7 in the same order).
__global__ void __launch_bounds__(256) k_math_eval(int fn, const double* __restrict__ x, double* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    double r;
    switch (fn) {
      case 0: r = fx::exp(v); break;
      case 1: r = fx::expm1(v); break;
      case 2: r = fx::log(v); break;
      case 3: r = fx::log1p(v); break;
      case 4: r = ::exp(v); break;
      case 5: r = ::expm1(v); break;
      case 6: r = ::log(v); break;
      default: r = ::log1p(v); break;
    }
    y[i] = r;
  }
}

void math_eval(int fn, const double* x, double* y, long long n, cudaStream_t s) {
  k_math_eval<<<grid_for(n), 256, 0, s>>>(fn, x, y, n);
}

}  // namespace rich
