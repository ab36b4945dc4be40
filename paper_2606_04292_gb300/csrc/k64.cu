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
            cudaStream_t s) {
  D::tail(dLs, dXs, l0, nl, P, model, nu1, nu2, cmax, crtol, gamma, gamma_levels, stats, s);
}

// ---------------------------------------------------------------------------
// Lagged state and history (eq. fully-bdf1; BDF2 reading: a = 3/(2 tau),
// history (4 theta^n - theta^{n-1}) / (2 tau), psi* = 2 psi^n - psi^{n-1}):
//   Kc = K(psi*),  g = a*history + xi psi*,  u = psi^n (initial iterate).
// ---------------------------------------------------------------------------
template <int MODEL>
__global__ void __launch_bounds__(256) k_prep_lagged(long long n, const double* __restrict__ psin,
                                                     const double* __restrict__ psinm1, const double* __restrict__ Ks,
                                                     double Ks_s, const double* __restrict__ p1f,
                                                     const double* __restrict__ p2f, Phys<double> P, int scheme,
                                                     double dt, double* Kc, double* g, double* u,
                                                     const double* thn_in, const double* thm_in, double* thn_out,
                                                     double* thm_out) {
  // thn_in / thm_in: theta(psi^n), theta(psi^{n-1}) kept from earlier FP64
  // evaluations (nullable: evaluate here, and keep them in *_out if given)
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double p1 = p1f ? p1f[i] : P.p1, p2 = p2f ? p2f[i] : P.p2;
    const double ks = Ks ? Ks[i] : Ks_s;
    const double pn = psin[i];
    double thn;
    if (thn_in) {
      thn = thn_in[i];
    } else {
      thn = theta_only_d<MODEL>(pn, p1, p2, P);
      if (thn_out) thn_out[i] = thn;
    }
    double ps, hist;
    if (scheme == 1) {
      ps = pn;
      hist = thn / dt;
    } else {
      const double pm = psinm1[i];
      double thm;
      if (thm_in) {
        thm = thm_in[i];
      } else {
        thm = theta_only_d<MODEL>(pm, p1, p2, P);
        if (thm_out) thm_out[i] = thm;
      }
      ps = 2.0 * pn - pm;
      hist = (4.0 * thn - thm) / (2.0 * dt);
    }
    Kc[i] = cond_d<MODEL>(ps, p1, p2, ks, P);
    g[i] = hist + P.xi * ps;
    u[i] = pn;
  }
}

// Gravity and boundary terms of g, and boundary face conductances:
//   gravity  -(M z)_i = (K_{i+e_z/2} - K_{i-e_z/2}) / h_z over interior faces,
//   Dirichlet (reading)  kb = (Kc_i + K(psi_b))/2,  g += 2 kb / h^2 (psi_b + z_b - z_i),
//   prescribed inflow q:  g += q / h,   free drainage:  g -= Kc_i / h_z.
template <int MODEL>
__global__ void __launch_bounds__(256) k_prep_rhs(Geom G, BcDev bc, const double* __restrict__ Ks, double Ks_s,
                                                  const double* __restrict__ p1f, const double* __restrict__ p2f,
                                                  Phys<double> P, const double* __restrict__ Kc, double* g,
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
    double gi = g[i];
    const double Ki = Kc[i];
    if (ii[v] + 1 < nn[v]) gi += 0.5 * (Ki + Kc[i + stride[v]]) / G.h[v];
    if (ii[v] > 0) gi -= 0.5 * (Ki + Kc[i - stride[v]]) / G.h[v];
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
          const double Kb = cond_d<MODEL>(val, p1, p2, Ks ? Ks[i] : Ks_s, P);
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

// restriction of a boundary-face array over the face's two in-plane axes
__global__ void __launch_bounds__(256) k_restrict_face(Geom F, Geom C, Xfer<double> X, int ax, const double* fine,
                                                       double* coarse) {
  int oa[2], k = 0;
  for (int a = 0; a < 3; ++a)
    if (a != ax) oa[k++] = a;
  const int nF[3] = {F.n0, F.n1, F.n2}, nC[3] = {C.n0, C.n1, C.n2};
  const long long nc = (long long)nC[oa[0]] * nC[oa[1]];
  for (long long J = blockIdx.x * (long long)blockDim.x + threadIdx.x; J < nc; J += (long long)gridDim.x * blockDim.x) {
    const int J0 = (int)(J % nC[oa[0]]), J1 = (int)(J / nC[oa[0]]);
    const int c0 = X.rc[oa[0]][J0], c1 = X.rc[oa[1]][J1];
    double s = 0.0;
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

// FP64 defect of the outer correction loop; hands the FP32 inner problem its
// right side r, its frozen state psi0 and a zero initial correction.
// th_in: theta(u) known already (the iterate is psi^n); otherwise theta(u) is
// evaluated and kept in th_out for the next step's history.
// theta(u) from th_in when given; else in FP64 (kept in th_out), or, with DD,
// in float-float arithmetic (accurate to ~1e-13, nothing kept).
template <int MODEL, bool DD>
__global__ void __launch_bounds__(256) k_outer_residual(Level<double> L, Phys<double> P, float* r32, float* psi0f,
                                                        float* delta, unsigned long long* norm,
                                                        const double* __restrict__ th_in, double* th_out) {
  __shared__ unsigned long long sm[33];
  unsigned long long mx = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.ncell;
       i += (long long)gridDim.x * blockDim.x) {
    int i0, i1, i2;
    cell_coords(L.n0, L.n1, i, i0, i1, i2);
    double mii, off;
    stencil(L, i, i0, i1, i2, L.u, mii, off);
    const double ui = L.u[i];
    double th;
    if (th_in) {
      th = th_in[i];
    } else if (DD) {
      th = theta_dd<MODEL>(ui, L.p1 ? L.p1[i] : P.p1, L.p2 ? L.p2[i] : P.p2, P);
    } else {
      th = theta_only_d<MODEL>(ui, L.p1 ? L.p1[i] : P.p1, L.p2 ? L.p2[i] : P.p2, P);
      th_out[i] = th;
    }
    double S, dS;
    sink_direct(ui, L.smax ? L.smax[i] : 0.0, P, S, dS);
    const double di = L.g[i] - (P.a * th + S + P.xi * ui + mii * ui - off);
    r32[i] = (float)di;
    psi0f[i] = (float)L.u[i];
    delta[i] = 0.0f;
    const unsigned long long b = nbits(di);
    mx = b > mx ? b : mx;
  }
  mx = block_max(mx, sm);
  if (threadIdx.x == 0) atomicMax(norm, mx);
}

__global__ void __launch_bounds__(256) k_apply_delta(double* u, const float* delta, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    u[i] += (double)delta[i];
}

void prep_lagged(const Geom& G, const double* psin, const double* psinm1, const double* Ks, double Ks_s,
                 const double* p1, const double* p2, const Phys<double>& P, int model, int scheme, double dt,
                 double* Kc, double* g, double* u, const double* thn_in, const double* thm_in, double* thn_out,
                 double* thm_out, cudaStream_t s) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const int b = grid_for(n);
  if (model == HAVERKAMP)
    k_prep_lagged<HAVERKAMP><<<b, 256, 0, s>>>(n, psin, psinm1, Ks, Ks_s, p1, p2, P, scheme, dt, Kc, g, u, thn_in,
                                               thm_in, thn_out, thm_out);
  else if (model == GARDNER)
    k_prep_lagged<GARDNER><<<b, 256, 0, s>>>(n, psin, psinm1, Ks, Ks_s, p1, p2, P, scheme, dt, Kc, g, u, thn_in,
                                             thm_in, thn_out, thm_out);
  else
    k_prep_lagged<VANGENUCHTEN><<<b, 256, 0, s>>>(n, psin, psinm1, Ks, Ks_s, p1, p2, P, scheme, dt, Kc, g, u, thn_in,
                                                  thm_in, thn_out, thm_out);
}

void prep_rhs(const Geom& G, const BcDev& bc, const double* Ks, double Ks_s, const double* p1, const double* p2,
              const Phys<double>& P, int model, const double* Kc, double* g, double* const kb[6], cudaStream_t s) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const int b = grid_for(n);
  if (model == HAVERKAMP)
    k_prep_rhs<HAVERKAMP><<<b, 256, 0, s>>>(G, bc, Ks, Ks_s, p1, p2, P, Kc, g, kb[0], kb[1], kb[2], kb[3], kb[4], kb[5]);
  else if (model == GARDNER)
    k_prep_rhs<GARDNER><<<b, 256, 0, s>>>(G, bc, Ks, Ks_s, p1, p2, P, Kc, g, kb[0], kb[1], kb[2], kb[3], kb[4], kb[5]);
  else
    k_prep_rhs<VANGENUCHTEN><<<b, 256, 0, s>>>(G, bc, Ks, Ks_s, p1, p2, P, Kc, g, kb[0], kb[1], kb[2], kb[3], kb[4],
                                               kb[5]);
}

void restrict_face64(const Geom& F, const Geom& C, const Xfer<double>& X, int axis, const double* fine,
                     double* coarse, cudaStream_t s) {
  const int nC[3] = {C.n0, C.n1, C.n2};
  long long nc = 1;
  for (int a = 0; a < 3; ++a)
    if (a != axis) nc *= nC[a];
  k_restrict_face<<<grid_for(nc), 256, 0, s>>>(F, C, X, axis, fine, coarse);
}

void sink_coef(const Geom& G, double Tp, double depth, double decay, double* smax, cudaStream_t s) {
  k_sink_coef<<<grid_for((long long)G.n0 * G.n1 * G.n2), 256, 0, s>>>(G, Tp, depth, decay, smax);
}

void to_float(const double* src, float* dst, long long n, cudaStream_t s) {
  k_to_float<<<grid_for(n), 256, 0, s>>>(src, dst, n);
}

template <bool DD>
static void outer_residual_t(const Level<double>& L, const Phys<double>& P, int model, float* r32, float* psi0f,
                             float* delta, unsigned long long* norm, const double* th_in, double* th_out,
                             cudaStream_t s) {
  const int b = grid_for(L.ncell);
  if (model == HAVERKAMP)
    k_outer_residual<HAVERKAMP, DD><<<b, 256, 0, s>>>(L, P, r32, psi0f, delta, norm, th_in, th_out);
  else if (model == GARDNER)
    k_outer_residual<GARDNER, DD><<<b, 256, 0, s>>>(L, P, r32, psi0f, delta, norm, th_in, th_out);
  else
    k_outer_residual<VANGENUCHTEN, DD><<<b, 256, 0, s>>>(L, P, r32, psi0f, delta, norm, th_in, th_out);
}

void outer_residual(const Level<double>& L, const Phys<double>& P, int model, float* r32, float* psi0f,
                    float* delta, unsigned long long* norm, const double* th_in, double* th_out, bool dd,
                    cudaStream_t s) {
  if (dd) outer_residual_t<true>(L, P, model, r32, psi0f, delta, norm, th_in, th_out, s);
  else outer_residual_t<false>(L, P, model, r32, psi0f, delta, norm, th_in, th_out, s);
}

template <int MODEL, bool DD>
__global__ void __launch_bounds__(256) k_soil_eval(long long n, const double* __restrict__ psi,
                                                   const double* __restrict__ Ks, double Ks_s,
                                                   const double* __restrict__ p1f, const double* __restrict__ p2f,
                                                   Phys<double> P, double* theta, double* K) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double p1 = p1f ? p1f[i] : P.p1, p2 = p2f ? p2f[i] : P.p2, x = psi[i];
    if (theta) theta[i] = DD ? theta_dd<MODEL>(x, p1, p2, P) : theta_only_d<MODEL>(x, p1, p2, P);
    if (K) {
      const double ks = Ks ? Ks[i] : Ks_s;
      K[i] = DD ? cond_dd<MODEL>(x, p1, p2, ks, P) : cond_d<MODEL>(x, p1, p2, ks, P);
    }
  }
}

template <bool DD>
static void soil_eval_t(long long n, const double* psi, const double* Ks, double Ks_s, const double* p1,
                        const double* p2, const Phys<double>& P, int model, double* theta, double* K,
                        cudaStream_t s) {
  const int b = grid_for(n);
  if (model == HAVERKAMP) k_soil_eval<HAVERKAMP, DD><<<b, 256, 0, s>>>(n, psi, Ks, Ks_s, p1, p2, P, theta, K);
  else if (model == GARDNER) k_soil_eval<GARDNER, DD><<<b, 256, 0, s>>>(n, psi, Ks, Ks_s, p1, p2, P, theta, K);
  else k_soil_eval<VANGENUCHTEN, DD><<<b, 256, 0, s>>>(n, psi, Ks, Ks_s, p1, p2, P, theta, K);
}

void soil_eval(long long n, const double* psi, const double* Ks, double Ks_s, const double* p1, const double* p2,
               const Phys<double>& P, int model, bool dd, double* theta, double* K, cudaStream_t s) {
  if (dd) soil_eval_t<true>(n, psi, Ks, Ks_s, p1, p2, P, model, theta, K, s);
  else soil_eval_t<false>(n, psi, Ks, Ks_s, p1, p2, P, model, theta, K, s);
}

void apply_delta(double* u, const float* delta, long long n, cudaStream_t s) {
  k_apply_delta<<<grid_for(n), 256, 0, s>>>(u, delta, n);
}

}  // namespace rich
