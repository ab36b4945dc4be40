// One implicit time step of a small grid without any device allocation.
//
// Who needs this: code that must not call cudaMalloc in the middle of its
// work -- an application whose memory pool already owns all of the device
// memory, a real-time loop that forbids allocator calls (they can block and
// synchronise the device), or a plug-in inside another GPU program that may
// only use memory handed to it.  Such callers pass
// device pointers for the state in and the state out; everything else the
// step needs (multigrid hierarchy, coefficients, transfer tables, norms)
// lives in one fixed array in the library's own device memory.
//
// The whole step runs in one thread block (a variant of the coarse-tail
// kernel that also does the per-step preparation and the stop loop), so the
// grid is limited to RICHARDS_NOALLOC_MAX_CELLS cells.
#include <cmath>
#include <cstring>

#include "kernels.cuh"
#include "richards.h"
#include "validate.h"

namespace rich {
namespace {

constexpr int NA_MAXLEV = 14;
constexpr long long NA_SCRATCH_DOUBLES = 262144;   // 2 MiB

// The fixed scratch array.  Every device that loads the library holds it
// until the process exits; all calls share it.
static __device__ __align__(256) double g_noalloc_scratch[NA_SCRATCH_DOUBLES];

struct NaLevel {
  Level<double> L;
  Xfer<double> X;          // tables to the next coarser level
  int *pc[3], *pj[3], *rc[3], *ri[3];
  double *pw[3], *rw[3];
  double* Kcw;             // writable views of the coefficient arrays
  double *p1w, *p2w, *smaxw;
  double* kbw[6];
};

struct NaPlan {
  int nlev, dim, model, scheme, max_cycles, nu1, nu2, cmax, gamma, gamma_levels, ordering;
  int ctx_mode;                    // 1: a context's hierarchy (its transfer tables, soil and sink arrays)
  double crtol, tol, dt, Lv, h[3];
  double slo[3], shi[3];           // prolongation ghost factors per axis
  int het_p1, het_p2, het_Ks, sink;
  double Ks, Tp, root_depth, root_decay;
  const double *psin, *psinm1, *Ks_field, *p1_field, *p2_field;
  double* psi_out;
  BcDev bc;
  Phys<double> P;
  double* stats;                   // [cycles, resid0, resid, status, updates]
  NaLevel lev[NA_MAXLEV];
};

// ---------------------------------------------------------------------------
// device pieces
// ---------------------------------------------------------------------------
// transfer tables of every level, built by the block
// (*overflow is set when a coarse cell would take more than RMAX fine
// contributors along an axis; ceil(n/2) coarsening gives at most 4)
__device__ void na_tables(const NaPlan& p, int* overflow) {
  for (int l = 0; l + 1 < p.nlev; ++l) {
    const NaLevel& F = p.lev[l];
    const NaLevel& C = p.lev[l + 1];
    const int nfa[3] = {F.L.n0, F.L.n1, F.L.n2}, nca[3] = {C.L.n0, C.L.n1, C.L.n2};
    for (int ax = 0; ax < 3; ++ax) {
      const int nf = nfa[ax], nc = nca[ax];
      for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        int idx[2];
        double w[2];
        int cnt;
        interp_row(nf, nc, i, p.slo[ax], p.shi[ax], idx, w, cnt);
        F.pc[ax][i] = cnt;
        for (int k = 0; k < 2; ++k) {
          F.pj[ax][2 * i + k] = k < cnt ? idx[k] : 0;
          F.pw[ax][2 * i + k] = k < cnt ? w[k] : 0.0;
        }
      }
      for (int J = threadIdx.x; J < nc; J += blockDim.x) {
        int cnt = 0;
        double s = 0.0;
        const int lo = nf == 1 ? 0 : (2 * J - 4 > 0 ? 2 * J - 4 : 0);
        const int hi = nf == 1 ? 0 : (2 * J + 4 < nf - 1 ? 2 * J + 4 : nf - 1);
        for (int i = lo; i <= hi; ++i) {
          int idx[2];
          double w[2];
          int c2;
          interp_row(nf, nc, i, 1.0, 1.0, idx, w, c2);
          for (int k = 0; k < c2; ++k)
            if (idx[k] == J) {
              if (cnt == RMAX) { *overflow = 1; continue; }
              F.ri[ax][RMAX * J + cnt] = i;
              F.rw[ax][RMAX * J + cnt] = w[k];
              ++cnt;
            }
        }
        for (int k = 0; k < cnt; ++k) s += F.rw[ax][RMAX * J + k];
        for (int k = 0; k < cnt; ++k) F.rw[ax][RMAX * J + k] /= s;
        F.rc[ax][J] = cnt;
      }
    }
  }
  __syncthreads();
}

// lagged state, Kc, history and the right side of the finest level
template <int MODEL>
__device__ void na_prepare(const NaPlan& p) {
  const NaLevel& F = p.lev[0];
  const Level<double>& L = F.L;
  const Phys<double>& P = p.P;
  for (long long i = threadIdx.x; i < L.ncell; i += blockDim.x) {
    const double p1 = p.p1_field ? p.p1_field[i] : P.p1, p2 = p.p2_field ? p.p2_field[i] : P.p2;
    if (!p.ctx_mode) {
      if (F.p1w) F.p1w[i] = p1;
      if (F.p2w) F.p2w[i] = p2;
    }
    const double pn = p.psin[i];
    const unsigned mi = mat_at<MODEL>(L.mat, i);
    const double thn = with_law<MODEL>(P, mi, [&](auto law, const Phys<double>& Q) {
      return theta_only_d<decltype(law)::value>(pn, p1, p2, Q);
    });
    double ps, hist;
    if (p.scheme == 1) {
      ps = pn;
      hist = thn / p.dt;
    } else {
      const double pm = p.psinm1[i];
      ps = P.lag ? pn : 2.0 * pn - pm;
      const double thm = with_law<MODEL>(P, mi, [&](auto law, const Phys<double>& Q) {
        return theta_only_d<decltype(law)::value>(pm, p1, p2, Q);
      });
      hist = (4.0 * thn - thm) / (2.0 * p.dt);
    }
    const double ks = p.Ks_field ? p.Ks_field[i] : p.Ks;
    F.Kcw[i] = with_law<MODEL>(P, mi, [&](auto law, const Phys<double>& Q) {
      return cond_d<decltype(law)::value>(ps, p1, p2, ks, Q);
    });
    L.g[i] = hist + P.xi * ps;
    L.u[i] = pn;
    if (F.smaxw && !p.ctx_mode) {
      int ii[3];
      cell_coords(L.n0, L.n1, i, ii[0], ii[1], ii[2]);
      const int v = p.dim - 1;
      const double lam = p.root_decay, D = p.root_depth;
      const double Z = lam * (1.0 - exp(-D / lam));
      const int nv = v == 0 ? L.n0 : (v == 1 ? L.n1 : L.n2);
      const double depth = p.Lv * (double)(2 * (nv - 1 - ii[v]) + 1) / (double)(2 * nv);
      F.smaxw[i] = depth <= D ? p.Tp * exp(-depth / lam) / Z : 0.0;
    }
  }
  __syncthreads();
  const int v = p.dim - 1;
  const int nn[3] = {L.n0, L.n1, L.n2};
  const long long stride[3] = {1, L.n0, (long long)L.n0 * L.n1};
  for (long long i = threadIdx.x; i < L.ncell; i += blockDim.x) {
    int ii[3];
    cell_coords(L.n0, L.n1, i, ii[0], ii[1], ii[2]);
    double gi = L.g[i];
    const double Ki = L.Kc[i];
    if (ii[v] + 1 < nn[v]) gi += 0.5 * (Ki + L.Kc[i + stride[v]]) / p.h[v];
    if (ii[v] > 0) gi -= 0.5 * (Ki + L.Kc[i - stride[v]]) / p.h[v];
    for (int ax = 0; ax < p.dim; ++ax)
      for (int side = 0; side < 2; ++side) {
        if (ii[ax] != (side ? nn[ax] - 1 : 0)) continue;
        const int f = 2 * ax + side;
        long long fc;
        if (ax == 0) fc = ii[1] + (long long)L.n1 * ii[2];
        else if (ax == 1) fc = ii[0] + (long long)L.n0 * ii[2];
        else fc = ii[0] + (long long)L.n0 * ii[1];
        const double h = p.h[ax];
        const int kind = p.bc.kind[f];
        const bool dir = kind == 0 && (!p.bc.mask[f] || p.bc.mask[f][fc]);
        const double val = p.bc.vfield[f] ? p.bc.vfield[f][fc] : p.bc.value[f];
        if (dir) {
          const double p1 = p.p1_field ? p.p1_field[i] : P.p1, p2 = p.p2_field ? p.p2_field[i] : P.p2;
          const double ks = p.Ks_field ? p.Ks_field[i] : p.Ks;
          const double kbv = with_law<MODEL>(P, mat_at<MODEL>(L.mat, i), [&](auto law, const Phys<double>& Q) {
            return cond_d<decltype(law)::value>(val, p1, p2, ks, Q);
          });
          const double k = 0.5 * (Ki + kbv);
          F.kbw[f][fc] = k;
          const double dz = (ax == v) ? (side ? 0.5 * h : -0.5 * h) : 0.0;
          gi += 2.0 * k / (h * h) * (val + dz);
        } else {
          F.kbw[f][fc] = 0.0;
          if (kind == 2) gi += val / h;
          else if (kind == 3) gi -= Ki / h;
        }
      }
    L.g[i] = gi;
  }
  __syncthreads();
  // coarse coefficients: restricted Kc, soil parameters, sink, face conductances
  for (int l = 0; l + 1 < p.nlev; ++l) {
    const NaLevel& Fl = p.lev[l];
    const NaLevel& Cl = p.lev[l + 1];
    for (long long J = threadIdx.x; J < Cl.L.ncell; J += blockDim.x) {
      int J0, J1, J2;
      cell_coords(Cl.L.n0, Cl.L.n1, J, J0, J1, J2);
      Cl.Kcw[J] = restrict_at(Fl.L, Fl.X, Fl.L.Kc, J0, J1, J2);
      if (p.ctx_mode) continue;      // (a context's coarse soil and sink arrays are set up already)
      if (Cl.p1w) Cl.p1w[J] = restrict_at(Fl.L, Fl.X, Fl.L.p1, J0, J1, J2);
      if (Cl.p2w) Cl.p2w[J] = restrict_at(Fl.L, Fl.X, Fl.L.p2, J0, J1, J2);
      if (Cl.smaxw) Cl.smaxw[J] = restrict_at(Fl.L, Fl.X, Fl.L.smax, J0, J1, J2);
    }
    const int nF[3] = {Fl.L.n0, Fl.L.n1, Fl.L.n2}, nC[3] = {Cl.L.n0, Cl.L.n1, Cl.L.n2};
    for (int f = 0; f < 2 * p.dim; ++f) {
      const int ax = f / 2;
      int oa[2], k = 0;
      for (int a = 0; a < 3; ++a)
        if (a != ax) oa[k++] = a;
      const long long nc = (long long)nC[oa[0]] * nC[oa[1]];
      for (long long J = threadIdx.x; J < nc; J += blockDim.x) {
        const int J0 = (int)(J % nC[oa[0]]), J1 = (int)(J / nC[oa[0]]);
        double s = 0.0;
        for (int a1 = 0; a1 < Fl.X.rc[oa[1]][J1]; ++a1)
          for (int a0 = 0; a0 < Fl.X.rc[oa[0]][J0]; ++a0)
            s += Fl.X.rw[oa[0]][RMAX * J0 + a0] * Fl.X.rw[oa[1]][RMAX * J1 + a1] *
                 Fl.L.kb[f][Fl.X.ri[oa[0]][RMAX * J0 + a0] + (long long)nF[oa[0]] * Fl.X.ri[oa[1]][RMAX * J1 + a1]];
        Cl.kbw[f][J] = s;
      }
    }
    __syncthreads();
  }
}

struct PlanLevels {
  const NaLevel* lev;
  __device__ const Level<double>& L(int l) const { return lev[l].L; }
  __device__ double restrict(int l, const double* fine, int J0, int J1, int J2) const {
    return restrict_at(lev[l].L, lev[l].X, fine, J0, J1, J2);
  }
  __device__ void restrict2(int l, const double* fa, const double* fb, int J0, int J1, int J2, double& a,
                            double& b) const {
    a = restrict(l, fa, J0, J1, J2);
    b = restrict(l, fb, J0, J1, J2);
  }
  __device__ double prolong(int l, int i0, int i1, int i2) const {
    return prolong_at(lev[l + 1].L, lev[l].X, i0, i1, i2);
  }
};

template <int MODEL>
__global__ void __launch_bounds__(TAIL_THREADS) k_small_step(const __grid_constant__ NaPlan p) {
  __shared__ unsigned long long sm[33];
  __shared__ int overflow;
  if (threadIdx.x == 0) overflow = 0;
  __syncthreads();
  if (!p.ctx_mode) na_tables(p, &overflow);   // ends with a barrier
  if (overflow) {                   // (uniform over the block)
    if (threadIdx.x == 0) {
      p.stats[0] = 0.0;
      p.stats[1] = p.stats[2] = 0.0;
      p.stats[3] = (double)RICH_EINVAL;
      p.stats[4] = 0.0;
    }
    return;
  }
  na_prepare<MODEL>(p);
  const Phys<double>& P = p.P;
  const double teff = 1.0 / P.a;
  double r = teff * block_defect_norm<double, FORM_DIRECT, MODEL>(p.lev[0].L, P, sm);
  const double r0 = r;
  int cycles = 0;
  unsigned long long updates = 0;
  while (!(r <= p.tol) && cycles < p.max_cycles && !isnan(r)) {
    block_cycle<double, FORM_DIRECT, MODEL>(PlanLevels{p.lev}, 0, p.nlev, P, p.nu1, p.nu2, p.cmax, p.crtol, p.gamma,
                                            p.gamma_levels, sm, updates, p.ordering);
    ++cycles;
    r = teff * block_defect_norm<double, FORM_DIRECT, MODEL>(p.lev[0].L, P, sm);
  }
  const Level<double>& F = p.lev[0].L;
  for (long long i = threadIdx.x; i < F.ncell; i += blockDim.x) p.psi_out[i] = F.u[i];
  if (threadIdx.x == 0) {
    p.stats[0] = cycles;
    p.stats[1] = r0;
    p.stats[2] = r;
    p.stats[3] = isnan(r) ? (double)RICH_ENAN : (r <= p.tol ? (double)RICH_OK : (double)RICH_ENOCONV);
    p.stats[4] = (double)updates;
  }
}

// Lays out the hierarchy of a small step over `base` (capacity doubles; base
// may be null to only count) and fills the plan.  lev0 (nullable): arrays of
// the finest level supplied by the caller (a context's own), so the step's
// lagged K, boundary conductances and right side land there.  Returns the
// doubles used, or -1 when they exceed the capacity.
long long build_plan(const richards_grid* grid, const richards_soil* soil, const richards_bc* bc,
                     const richards_sink* sink, const richards_opts& o, double dt, int scheme, const double* psi_n,
                     const double* psi_prev, double* psi_out, double* base, long long capacity, const SmallCtx* cx,
                     int ordering, NaPlan& p) {
  std::memset(&p, 0, sizeof(p));
  long long used = 0;
  bool overflow = false;
  auto take = [&](long long ndoubles) -> double* {
    const long long n = (ndoubles + 31) / 32 * 32;   // keep 256-byte alignment
    if (used + n > capacity) { overflow = true; return base; }
    double* q = base ? base + used : nullptr;
    used += n;
    return q;
  };
  p.stats = take(8);
  int n[NA_MAXLEV][3];
  for (int a = 0; a < 3; ++a) n[0][a] = grid->n[a];
  int nlev = 1;
  for (;;) {
    const int mx = n[nlev - 1][0] > n[nlev - 1][1] ? (n[nlev - 1][0] > n[nlev - 1][2] ? n[nlev - 1][0] : n[nlev - 1][2])
                                                   : (n[nlev - 1][1] > n[nlev - 1][2] ? n[nlev - 1][1] : n[nlev - 1][2]);
    if (mx <= o.coarsest_max_n || (o.max_levels > 0 && nlev >= o.max_levels) || nlev >= NA_MAXLEV) break;
    for (int a = 0; a < 3; ++a) n[nlev][a] = n[nlev - 1][a] > 1 ? (n[nlev - 1][a] + 1) / 2 : 1;
    ++nlev;
  }
  if (cx) {
    if (cx->nlev != nlev) return -1;
    p.ctx_mode = 1;
  }
  p.nlev = nlev;
  p.dim = grid->dim;
  const bool het_p1 = soil->p1_field != nullptr, het_p2 = soil->p2_field != nullptr;
  for (int l = 0; l < nlev; ++l) {
    NaLevel& H = p.lev[l];
    Level<double>& L = H.L;
    if (cx) {                        // every array and table of the context's level
      L = cx->L[l];
      H.X = cx->X[l];
      H.Kcw = const_cast<double*>(L.Kc);
      for (int f = 0; f < 6; ++f) H.kbw[f] = const_cast<double*>(L.kb[f]);
      continue;
    }
    L.dim = grid->dim;
    L.n0 = n[l][0]; L.n1 = n[l][1]; L.n2 = n[l][2];
    L.ncell = (long long)L.n0 * L.n1 * L.n2;
    for (int a = 0; a < 3; ++a) {
      const double h = a < grid->dim ? grid->L[a] / n[l][a] : 1.0;
      L.ih2[a] = a < grid->dim ? 1.0 / (h * h) : 0.0;
    }
    L.u = take(L.ncell); L.ubar = take(L.ncell); L.g = take(L.ncell); L.d = take(L.ncell);
    H.Kcw = take(L.ncell);
    H.p1w = het_p1 ? take(L.ncell) : nullptr;
    H.p2w = het_p2 ? take(L.ncell) : nullptr;
    H.smaxw = sink->enabled ? take(L.ncell) : nullptr;
    for (int f = 0; f < 6; ++f) H.kbw[f] = f < 2 * grid->dim ? take(L.ncell / n[l][f / 2]) : nullptr;
    L.Kc = H.Kcw;
    L.p1 = H.p1w; L.p2 = H.p2w; L.smax = H.smaxw;
    L.psi0 = nullptr;
    for (int f = 0; f < 6; ++f) L.kb[f] = H.kbw[f];
    if (l + 1 < nlev)
      for (int a = 0; a < 3; ++a) {
        const int nf = n[l][a], nc = n[l + 1][a];
        H.pc[a] = (int*)take((nf + 1) / 2);
        H.pj[a] = (int*)take(nf);
        H.pw[a] = take(2LL * nf);
        H.rc[a] = (int*)take((nc + 1) / 2);
        H.ri[a] = (int*)take((RMAX * (long long)nc + 1) / 2);
        H.rw[a] = take(RMAX * (long long)nc);
        H.X.pc[a] = H.pc[a]; H.X.pj[a] = H.pj[a]; H.X.pw[a] = H.pw[a];
        H.X.rc[a] = H.rc[a]; H.X.ri[a] = H.ri[a]; H.X.rw[a] = H.rw[a];
      }
  }
  if (overflow) return -1;

  p.model = soil->model;
  p.scheme = (scheme == 2 && psi_prev) ? 2 : 1;
  p.max_cycles = o.max_cycles;
  p.nu1 = o.nu1;
  p.nu2 = o.nu2;
  p.cmax = o.coarse_max_sweeps;
  p.gamma = o.cycle_gamma;
  p.gamma_levels = o.gamma_levels;
  p.crtol = o.coarse_rtol;
  p.tol = o.tol;
  p.dt = dt;
  p.ordering = ordering;
  for (int a = 0; a < 3; ++a) {
    p.h[a] = a < grid->dim ? grid->L[a] / grid->n[a] : 1.0;
    p.slo[a] = p.shi[a] = 1.0;
    if (a < grid->dim) {
      if (bc->kind[2 * a] == RICH_BC_DIRICHLET && !bc->mask_field[2 * a]) p.slo[a] = -1.0;
      if (bc->kind[2 * a + 1] == RICH_BC_DIRICHLET && !bc->mask_field[2 * a + 1]) p.shi[a] = -1.0;
    }
  }
  p.Lv = grid->L[grid->dim - 1];
  p.Ks = soil->Ks;
  p.Tp = sink->Tp;
  p.root_depth = sink->root_depth;
  p.root_decay = sink->root_decay;
  p.psin = psi_n;
  p.psinm1 = psi_prev;
  p.Ks_field = soil->Ks_field;
  p.p1_field = soil->p1_field;
  p.p2_field = soil->p2_field;
  p.psi_out = psi_out;
  for (int f = 0; f < 6; ++f) {
    p.bc.kind[f] = f < 2 * grid->dim ? bc->kind[f] : RICH_BC_NOFLUX;
    p.bc.value[f] = f < 2 * grid->dim ? bc->value[f] : 0.0;
    p.bc.vfield[f] = f < 2 * grid->dim ? bc->value_field[f] : nullptr;
    p.bc.mask[f] = f < 2 * grid->dim ? bc->mask_field[f] : nullptr;
  }
  Phys<double>& P = p.P;
  P.a = p.scheme == 1 ? 1.0 / dt : 1.5 / dt;
  P.xi = o.xi;
  P.kappa = o.kappa_mode == 0 ? o.kappa : 0.0;
  P.ts = soil->theta_s;
  P.tr = soil->theta_r;
  P.p1 = soil->p1; P.p2 = soil->p2; P.p3 = soil->p3; P.p4 = soil->p4;
  P.h1 = sink->h1; P.h2 = sink->h2; P.h3 = sink->h3; P.h4 = sink->h4;
  P.newton_k = o.newton_iters;
  P.sink = sink->enabled;
  P.lag = o.bdf2_lag;
  if (cx) P.mats = cx->mats;
  return used;
}

void launch_plan(const NaPlan& p, cudaStream_t s) {
  if (p.model == RICH_HAVERKAMP) k_small_step<HAVERKAMP><<<1, TAIL_THREADS, 0, s>>>(p);
  else if (p.model == RICH_GARDNER) k_small_step<GARDNER><<<1, TAIL_THREADS, 0, s>>>(p);
  else if (p.model == COMPOSITE) k_small_step<COMPOSITE><<<1, TAIL_THREADS, 0, s>>>(p);
  else k_small_step<VANGENUCHTEN><<<1, TAIL_THREADS, 0, s>>>(p);
}

// device address of the scratch array, looked up once per device
constexpr int NA_MAXDEV = 64;
double* g_scratch_addr[NA_MAXDEV] = {nullptr};

}  // namespace

richards_status small_step(const richards_grid* grid, const richards_soil* soil, const richards_bc* bc,
                           const richards_sink* sink, const richards_opts* opts, double dt, int scheme,
                           const double* psi_n, const double* psi_prev, double* psi_out, double* stats_dev,
                           const SmallCtx* cx, int ordering, double* stats_out, cudaStream_t s) {
  NaPlan p;
  if (build_plan(grid, soil, bc, sink, *opts, dt, scheme, psi_n, psi_prev, psi_out, stats_dev, 32, cx, ordering, p) <
      0)
    return RICH_EINVAL;
  launch_plan(p, s);
  if (cudaGetLastError() != cudaSuccess) return RICH_ECUDA;
  if (cudaMemcpyAsync(stats_out, p.stats, 5 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return RICH_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return RICH_ECUDA;
  return RICH_OK;
}

}  // namespace rich

extern "C" richards_status richards_step_small_noalloc(const richards_grid* grid, const richards_soil* soil,
                                                       const richards_bc* bc, const richards_sink* sink,
                                                       const richards_opts* opts, double dt, int scheme,
                                                       const double* psi_n, const double* psi_prev, double* psi_out,
                                                       richards_step_info* info, void* stream) {
  using namespace rich;
  if (!grid || !soil || !bc || !sink || !opts || !psi_n || !psi_out) return RICH_EINVAL;
  if (grid->dim < 1 || grid->dim > 3) return RICH_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (grid->n[a] < 1 || (a >= grid->dim && grid->n[a] != 1)) return RICH_EINVAL;
    if (a < grid->dim && !(grid->L[a] > 0.0 && std::isfinite(grid->L[a]))) return RICH_EINVAL;
  }
  const long long N = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  if (N > RICHARDS_NOALLOC_MAX_CELLS) return RICH_EINVAL;          // grid larger than the fixed scratch
  const richards_opts& o = *opts;
  if (!(dt > 0.0) || !std::isfinite(dt) || (scheme != 1 && scheme != 2) || o.nu1 < 0 || o.nu2 < 0 ||
      o.coarse_max_sweeps < 1 || o.max_cycles < 0 || o.coarsest_max_n < 1 || !(o.tol > 0.0) ||
      o.newton_iters < 0 || o.newton_iters > 200 || (o.kappa_mode != 0 && o.kappa_mode != 2) ||
      !(o.xi >= 0.0) || !(o.kappa >= 0.0) || o.cycle_gamma < 1 || o.cycle_gamma > 3 || o.gamma_levels < 0 ||
      (o.bdf2_lag != 0 && o.bdf2_lag != 1))
    return RICH_EINVAL;
  // the same checks as richards_set_soil / set_bc / set_sink (the fields are
  // device arrays here and are not read on the host)
  if (law_error(soil->model, soil->Ks, soil->theta_s, soil->theta_r, soil->p1, soil->p2, soil->p3, soil->p4,
                soil->p1_field != nullptr, soil->p2_field != nullptr) ||
      bc_error(*bc, grid->dim) || sink_error(*sink))
    return RICH_EINVAL;

  // set-up, once per device: the device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAXDEV) return RICH_ECUDA;
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) return RICH_ECUDA;
    g_scratch_addr[dev] = (double*)ptr;
  }
  // the hierarchy carved out of the scratch array (red-black sweeps)
  NaPlan p;
  if (build_plan(grid, soil, bc, sink, o, dt, scheme, psi_n, psi_prev, psi_out, g_scratch_addr[dev],
                 NA_SCRATCH_DOUBLES, nullptr, 1, p) < 0)
    return RICH_EINVAL;   // hierarchy larger than the fixed scratch

  cudaStream_t s = (cudaStream_t)stream;
  launch_plan(p, s);
  if (cudaGetLastError() != cudaSuccess) return RICH_ECUDA;
  double stats[5];
  if (cudaMemcpyAsync(stats, p.stats, sizeof(stats), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RICH_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return RICH_ECUDA;
  if (info) {
    info->cycles = (int)stats[0];
    info->outer_iters = 0;
    info->scheme_used = p.scheme;
    info->resid0 = stats[1];
    info->resid = stats[2];
    info->cell_updates = (long long)stats[4];
    info->mass_defect = NAN;    // not computed on this path
    info->err_bound = NAN;
  }
  return (richards_status)(int)stats[3];
}
