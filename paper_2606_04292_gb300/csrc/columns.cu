// Batched independent soil columns in one persistent launch.
//
// Each thread block takes columns from a device work queue (one atomic
// counter over a longest-first order) and runs every time step of its column:
// per-step preparation and the defect of the outer correction loop in
// float-float arithmetic on the column's slices of global arrays, and the
// FP32 FAS cycles of the inner correction problem with the whole multigrid
// hierarchy of the column in shared memory.  Columns are 1D (axis 0 is the vertical), of any length up
// to RICHARDS_COLUMN_MAX_CELLS, each with its own scalar soil parameters and
// boundary conditions; one soil law for the whole batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "richards.h"
#include "validate.h"

namespace rich {
namespace {

constexpr int COL_MAXLEV = 14;
constexpr int COL_THREADS_MAX = 512;
constexpr int COL_ARRAYS = 7;      // u, ubar, g, d, Kc, psi0, smax per level (FP32)

struct ColDesc {
  long long off;                   // first cell in the packed arrays
  int n;                           // cells
  int bc_kind[2];                  // bottom, top
  double bc_val[2];
  double Lz, Ks, ts, tr, p1, p2, p3, p4;
};

struct ColArgs {
  const ColDesc* cols;
  const int* order;                // processing order (longest first)
  int ncol;
  int begin, end;                  // this launch's columns: order[begin, end)
  int* queue;                      // work counter, zero before the launch
  int* thn_valid;                  // per column: thn holds theta(psi^n)
  double *psin, *psinm1, *u, *g, *Kc, *thn, *thcur, *smax;
  int* have_prev;
  int *st_status, *st_cycles, *st_outer;
  double* st_resid;
  unsigned long long* st_updates;
  int sink;
  int fp64;                        // outer layer: 1 FP64 (precision 2), 0 float-float
  double h1, h2, h3, h4, xi, kappa, tol, inner_rtol, crtol, dt;
  int newton_k, max_outer, inner_cycles, nu1, nu2, cmax, gamma, gamma_levels, coarsest_max_n, scheme, nsteps, lag,
      model;
};

// The interpolation row of fine cell i (the same reading as the tables of the
// multi-dimensional path: coarse coordinate ((2i+1) nc - nf)/(2 nf), a ghost
// beyond an end folded into the end cell with factor slo/shi) in FP32 and
// 32-bit integers: columns have at most RICHARDS_COLUMN_MAX_CELLS cells.
__device__ __forceinline__ void interp_row_f(int nf, int nc, int i, float slo, float shi, int* idx, float* w,
                                             int& cnt) {
  cnt = 0;
  auto add = [&](int j, float wt) {
    if (wt == 0.0f) return;
    for (int k = 0; k < cnt; ++k)
      if (idx[k] == j) { w[k] += wt; return; }
    idx[cnt] = j;
    w[cnt] = wt;
    ++cnt;
  };
  if (nf == 1) { add(0, 1.0f); return; }
  const int num = (2 * i + 1) * nc - nf, den = 2 * nf;
  // floor(num / den) through the FP32 quotient, then corrected: |num| and den
  // are below 2^24 (exact in FP32) and the quotient's floor is off by at most
  // one, so one test each way gives the exact integer floor
  int J0 = (int)floorf(__fdividef((float)num, (float)den));
  if (J0 * den > num) --J0;
  else if ((J0 + 1) * den <= num) ++J0;
  const float wt = (float)(num - J0 * den) / (float)den;
  const int J1 = J0 + 1;
  if (J0 < 0) add(0, (1.0f - wt) * slo); else add(J0, 1.0f - wt);
  if (J1 >= nc) add(nc - 1, wt * shi); else add(J1, wt);
}

// 1D hierarchy of one column in shared memory; transfer weights computed on
// the fly (columns have arbitrary lengths) in FP32: R is the transpose of the
// constant-extrapolation P with rows normalised to 1, P folds the ghost with
// slo/shi (-1 on a Dirichlet end).
struct ColumnLevels {
  const Level<float>* Ls;
  float slo, shi;
  __device__ const Level<float>& L(int l) const { return Ls[l]; }
  // the taps of coarse row J0: fine indices ri, weights rw (cnt of them) and
  // the inverse of their sum
  __device__ int taps(int l, int J0, int* ri, float* rw, float& inv) const {
    const int nf = Ls[l].n0, nc = Ls[l + 1].n0;
    int cnt = 0;
    // (nc = ceil(nf/2): a fine cell i reaches coarse rows floor(t), floor(t) + 1
    // with t = ((2i+1) nc - nf) / (2 nf), so the cells of row J0 lie in
    // [2 J0 - 2, 2 J0 + 2]; checked for every nf up to 2048)
    const int lo = nf == 1 ? 0 : max(0, 2 * J0 - 2), hi = nf == 1 ? 0 : min(nf - 1, 2 * J0 + 2);
    for (int i = lo; i <= hi; ++i) {
      int idx[2];
      float w[2];
      int c2;
      interp_row_f(nf, nc, i, 1.0f, 1.0f, idx, w, c2);
      for (int k = 0; k < c2; ++k)
        if (idx[k] == J0 && cnt < RMAX) { ri[cnt] = i; rw[cnt] = w[k]; ++cnt; }
    }
    float s = 0.0f;
    for (int k = 0; k < cnt; ++k) s += rw[k];
    inv = 1.0f / s;
    return cnt;
  }
  __device__ float restrict(int l, const float* fine, int J0, int, int) const {
    int ri[RMAX];
    float rw[RMAX], inv;
    const int cnt = taps(l, J0, ri, rw, inv);
    float acc = 0.0f;
    for (int k = 0; k < cnt; ++k) acc += rw[k] * inv * fine[ri[k]];
    return acc;
  }
  // two arrays through one computation of the taps (the same sums as two
  // restrict calls)
  __device__ void restrict2(int l, const float* fa, const float* fb, int J0, int, int, float& a, float& b) const {
    int ri[RMAX];
    float rw[RMAX], inv;
    const int cnt = taps(l, J0, ri, rw, inv);
    float sa = 0.0f, sb = 0.0f;
    for (int k = 0; k < cnt; ++k) {
      sa += rw[k] * inv * fa[ri[k]];
      sb += rw[k] * inv * fb[ri[k]];
    }
    a = sa;
    b = sb;
  }
  __device__ float prolong(int l, int i0, int, int) const {
    const Level<float>& C = Ls[l + 1];
    int idx[2];
    float w[2];
    int cnt;
    interp_row_f(Ls[l].n0, C.n0, i0, slo, shi, idx, w, cnt);
    float acc = 0.0f;
    for (int k = 0; k < cnt; ++k) acc += w[k] * (C.u[idx[k]] - C.ubar[idx[k]]);
    return acc;
  }
};

template <int MODEL>
__device__ void column_solve(const ColArgs& A, int c, float* smem, Level<float>* Ls, int* s_nl, double* kb64,
                             unsigned long long* sm) {
  const ColDesc D = A.cols[c];
  const int n = D.n;
  const long long off = D.off;
  const double h = D.Lz / n;
  // hierarchy in shared memory
  if (threadIdx.x == 0) {
    int nn = n, l = 0;
    float* p = smem;
    for (;;) {
      Level<float>& V = Ls[l];
      V.dim = 1; V.n0 = nn; V.n1 = 1; V.n2 = 1; V.ncell = nn;
      const double hl = D.Lz / nn;
      V.ih2[0] = (float)(1.0 / (hl * hl)); V.ih2[1] = 0.0f; V.ih2[2] = 0.0f;
      V.u = p; V.ubar = p + nn; V.g = p + 2 * nn; V.d = p + 3 * nn;
      V.Kc = p + 4 * nn; V.psi0 = p + 5 * nn; V.smax = A.sink ? p + 6 * nn : nullptr;
      V.p1 = nullptr; V.p2 = nullptr;
      V.mat = nullptr; V.cs = 0;
      p += COL_ARRAYS * nn;
      V.kb[0] = p; V.kb[1] = p + 1;
      V.kb[2] = V.kb[3] = V.kb[4] = V.kb[5] = nullptr;
      p += 2;
      ++l;
      if (nn <= A.coarsest_max_n || l >= COL_MAXLEV) break;
      nn = (nn + 1) / 2;
    }
    *s_nl = l;
  }
  __syncthreads();
  const int nl = *s_nl;
  const ColumnLevels lv{Ls, (D.bc_kind[0] == RICH_BC_DIRICHLET) ? -1.0f : 1.0f,
                        (D.bc_kind[1] == RICH_BC_DIRICHLET) ? -1.0f : 1.0f};
  // FP64 view of the finest level on the column's slices of global memory
  Level<double> G{};
  G.dim = 1; G.n0 = n; G.n1 = 1; G.n2 = 1; G.ncell = n;
  G.ih2[0] = 1.0 / (h * h);
  G.u = A.u + off; G.g = A.g + off; G.Kc = A.Kc + off;
  G.smax = A.sink ? A.smax + off : nullptr;
  G.kb[0] = kb64; G.kb[1] = kb64 + 1;
  Phys<double> P64{};
  P64.xi = A.xi; P64.kappa = A.kappa; P64.ts = D.ts; P64.tr = D.tr;
  P64.p1 = D.p1; P64.p2 = D.p2; P64.p3 = D.p3; P64.p4 = D.p4;
  P64.h1 = A.h1; P64.h2 = A.h2; P64.h3 = A.h3; P64.h4 = A.h4;
  P64.newton_k = A.newton_k; P64.sink = A.sink; P64.lag = A.lag;
  Phys<float> P32{};
  P32.xi = (float)A.xi; P32.kappa = (float)A.kappa; P32.ts = (float)D.ts; P32.tr = (float)D.tr;
  P32.p1 = (float)D.p1; P32.p2 = (float)D.p2; P32.p3 = (float)D.p3; P32.p4 = (float)D.p4;
  P32.h1 = (float)A.h1; P32.h2 = (float)A.h2; P32.h3 = (float)A.h3; P32.h4 = (float)A.h4;
  P32.newton_k = A.newton_k; P32.sink = A.sink; P32.lag = A.lag;
  double* psin = A.psin + off;
  double* psinm1 = A.psinm1 + off;
  double* thn = A.thn + off;
  double* thcur = A.thcur + off;
  // sink coefficients of every level (FP32)
  if (A.sink) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) const_cast<float*>(Ls[0].smax)[i] = (float)A.smax[off + i];
    __syncthreads();
    for (int l = 0; l + 1 < nl; ++l) {
      for (int J = threadIdx.x; J < Ls[l + 1].n0; J += blockDim.x)
        const_cast<float*>(Ls[l + 1].smax)[J] = lv.restrict(l, Ls[l].smax, J, 0, 0);
      __syncthreads();
    }
  }
  int status = RICH_OK, cyc_total = 0, outer_total = 0;
  double resid = 0.0;
  unsigned long long updates = 0;
  int have_prev = A.have_prev[c];
  int th_valid = A.thn_valid[c];
  for (int step = 0; step < A.nsteps && status != RICH_ENAN; ++step) {
    const int scheme = (A.scheme == 2 && have_prev) ? 2 : 1;
    const double a = scheme == 1 ? 1.0 / A.dt : 1.5 / A.dt;
    P64.a = a;
    P32.a = (float)a;
    const DDPhys Q = make_ddphys_dev(P64);
    const dd Ks = dd_split(D.Ks);
    const dd hist_scale = dd_split(scheme == 1 ? 1.0 / A.dt : 1.0 / (2.0 * A.dt));
    // ---- per-step preparation (float-float, or FP64 with the FP64 outer
    // layer): lagged K, history, u = psi^n
    for (int i = threadIdx.x; i < n && A.fp64; i += blockDim.x) {
      const double pnd = psin[i];
      double th;
      if (th_valid) {
        th = thn[i];
      } else {
        th = theta_only_d<MODEL>(pnd, D.p1, D.p2, P64);
        thn[i] = th;
      }
      double ps, hist;
      if (scheme == 1) {
        ps = pnd;
        hist = th / A.dt;
      } else {
        const double pm = psinm1[i];
        ps = A.lag ? pnd : 2.0 * pnd - pm;
        hist = (4.0 * th - theta_only_d<MODEL>(pm, D.p1, D.p2, P64)) / (2.0 * A.dt);
      }
      A.Kc[off + i] = cond_d<MODEL>(ps, D.p1, D.p2, D.Ks, P64);
      G.g[i] = hist + A.xi * ps;
      G.u[i] = pnd;
    }
    for (int i = threadIdx.x; i < n && !A.fp64; i += blockDim.x) {
      const double pnd = psin[i];
      const dd pn = dd_split(pnd);
      dd th;
      if (th_valid) {
        th = dd_split(thn[i]);
      } else {
        th = theta_x<MODEL>(pn, Q.p1, Q.p2, Q, P64);
        thn[i] = dd_join(th);
      }
      dd ps, hist;
      if (scheme == 1) {
        ps = pn;
        hist = dd_mul(th, hist_scale);
      } else {
        const dd pm = dd_split(psinm1[i]);
        ps = A.lag ? pn : dd_sub(mk(2.0f * pn.hi, 2.0f * pn.lo), pm);
        hist = dd_mul(dd_sub(mk(4.0f * th.hi, 4.0f * th.lo), theta_x<MODEL>(pm, Q.p1, Q.p2, Q, P64)), hist_scale);
      }
      A.Kc[off + i] = dd_join(cond_x<MODEL>(ps, Q.p1, Q.p2, Ks, Q, P64));
      G.g[i] = dd_join(dd_add(hist, dd_mul(Q.xi, ps)));
      G.u[i] = pnd;
    }
    th_valid = 1;
    __syncthreads();
    // gravity and boundary terms (axis 0 is vertical; face 0 bottom, 1 top)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double gi = G.g[i];
      const double Ki = G.Kc[i];
      if (i + 1 < n) gi += 0.5 * (Ki + G.Kc[i + 1]) / h;
      if (i > 0) gi -= 0.5 * (Ki + G.Kc[i - 1]) / h;
      for (int side = 0; side < 2; ++side) {
        if (i != (side ? n - 1 : 0)) continue;
        const int kind = D.bc_kind[side];
        const double val = D.bc_val[side];
        if (kind == RICH_BC_DIRICHLET) {
          const double k = 0.5 * (Ki + cond_d<MODEL>(val, D.p1, D.p2, D.Ks, P64));
          kb64[side] = k;
          gi += 2.0 * k / (h * h) * (val + (side ? 0.5 * h : -0.5 * h));
        } else {
          kb64[side] = 0.0;
          if (kind == RICH_BC_FLUX) gi += val / h;
          else if (kind == RICH_BC_FREE_DRAINAGE) gi -= Ki / h;
        }
      }
      G.g[i] = gi;
    }
    __syncthreads();
    // FP32 coefficients of the inner problem on every level
    for (int i = threadIdx.x; i < n; i += blockDim.x) const_cast<float*>(Ls[0].Kc)[i] = (float)G.Kc[i];
    if (threadIdx.x < 2) const_cast<float*>(Ls[0].kb[threadIdx.x])[0] = (float)kb64[threadIdx.x];
    __syncthreads();
    for (int l = 0; l + 1 < nl; ++l) {
      for (int J = threadIdx.x; J < Ls[l + 1].n0; J += blockDim.x)
        const_cast<float*>(Ls[l + 1].Kc)[J] = lv.restrict(l, Ls[l].Kc, J, 0, 0);
      if (threadIdx.x < 2) const_cast<float*>(Ls[l + 1].kb[threadIdx.x])[0] = Ls[l].kb[threadIdx.x][0];
      __syncthreads();
    }
    // ---- defect correction around FP32 cycles; the defect in float-float,
    // interior fluxes in difference form m_f (u_i - u_j)
    const double teff = 1.0 / a;
    const dd hs = dd_split(0.5 / (h * h)), s2 = dd_split(2.0 / (h * h));
    const dd db0 = dd_mul(dd_split(kb64[0]), s2), db1 = dd_mul(dd_split(kb64[1]), s2);
    int outer = 0;
    bool fresh = false;
    // the FP64 outer layer's deciding defect: the expression of the grid
    // path's FP64 defect (interior fluxes in difference form), theta(u) kept
    // for the history when u moved
    auto defect64 = [&]() -> double {
      unsigned long long mx = 0;
      const double ih2 = 1.0 / (h * h), hs2 = 0.5 * ih2;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double ui = G.u[i], Ki = G.Kc[i];
        double flux = 0.0, db = 0.0;
        if (i > 0) flux += (Ki + G.Kc[i - 1]) * hs2 * (ui - G.u[i - 1]);
        else db += 2.0 * kb64[0] * ih2;
        if (i + 1 < n) flux += (Ki + G.Kc[i + 1]) * hs2 * (ui - G.u[i + 1]);
        else db += 2.0 * kb64[1] * ih2;
        double th;
        if (outer == 0) {
          th = thn[i];
        } else {
          th = theta_only_d<MODEL>(ui, D.p1, D.p2, P64);
          thcur[i] = th;
        }
        double S, dS;
        sink_direct(ui, G.smax ? G.smax[i] : 0.0, P64, S, dS);
        const double di = G.g[i] - ((a * th + S) + (A.xi + db) * ui + flux);
        Ls[0].g[i] = (float)di;
        const_cast<float*>(Ls[0].psi0)[i] = (float)ui;
        Ls[0].u[i] = 0.0f;
        const unsigned long long b = nbits(di);
        mx = b > mx ? b : mx;
      }
      return __longlong_as_double((long long)block_max(mx, sm));
    };
    bool use64 = false;                  // (the grid path's hand-over to FP64 defects)
    double r_ff = INFINITY;
    for (;;) {
      unsigned long long mx = 0;
      for (int i = threadIdx.x; i < n && !use64; i += blockDim.x) {
        const dd ui = dd_split(G.u[i]), Ki = dd_split(G.Kc[i]);
        dd flux = mk(0.0f), db = mk(0.0f);
        if (i > 0)
          flux = dd_add(flux, dd_mul(dd_mul(dd_add(Ki, dd_split(G.Kc[i - 1])), hs), dd_sub(ui, dd_split(G.u[i - 1]))));
        else
          db = dd_add(db, db0);
        if (i + 1 < n)
          flux = dd_add(flux, dd_mul(dd_mul(dd_add(Ki, dd_split(G.Kc[i + 1])), hs), dd_sub(ui, dd_split(G.u[i + 1]))));
        else
          db = dd_add(db, db1);
        dd th;
        if (outer == 0) {
          th = dd_split(thn[i]);
        } else {
          th = theta_x<MODEL>(ui, Q.p1, Q.p2, Q, P64);
          if (!A.fp64) thcur[i] = dd_join(th);     // (FP64 outer: from the FP64 defect)
        }
        const dd S = G.smax ? sink_x(ui, dd_split(G.smax[i]), Q) : mk(0.0f);
        dd N = dd_add(dd_mul(Q.a, th), S);
        N = dd_add(N, dd_mul(dd_add(Q.xi, db), ui));
        N = dd_add(N, flux);
        const float r = dd_float(dd_sub(dd_split(G.g[i]), N));
        Ls[0].g[i] = r;
        const_cast<float*>(Ls[0].psi0)[i] = dd_float(ui);
        Ls[0].u[i] = 0.0f;
        const unsigned long long b = nbits(r);
        mx = b > mx ? b : mx;
      }
      fresh = outer > 0;
      double nrm = 0.0;
      if (!use64) {
        nrm = (double)__uint_as_float((unsigned)block_max(mx, sm));
        resid = teff * nrm;
        const double prev = r_ff;
        r_ff = resid;
        use64 = A.fp64 && !isnan(resid) && (!(resid > A.tol) || outer >= A.max_outer || resid > 0.5 * prev);
      }
      if (use64) {
        nrm = defect64();                     // the FP64 defect decides
        resid = teff * nrm;
      }
      if (!(resid > A.tol) || isnan(resid)) break;
      if (outer >= A.max_outer) { status = RICH_ENOCONV; break; }
      for (int l = 0; l + 1 < nl; ++l) {
        for (int J = threadIdx.x; J < Ls[l + 1].n0; J += blockDim.x)
          const_cast<float*>(Ls[l + 1].psi0)[J] = lv.restrict(l, Ls[l].psi0, J, 0, 0);
        __syncthreads();
      }
      const float rin0 = (float)nrm;
      for (int k = 0; k < A.inner_cycles; ++k) {
        block_cycle<float, FORM_DELTA, MODEL>(lv, 0, nl, P32, A.nu1, A.nu2, A.cmax, (float)A.crtol, A.gamma,
                                              A.gamma_levels, sm, updates);
        ++cyc_total;
        if (A.inner_rtol > 0.0 && k + 1 < A.inner_cycles) {
          const float rin = block_defect_norm<float, FORM_DELTA, MODEL>(Ls[0], P32, sm);
          if (rin <= (float)A.inner_rtol * rin0) break;
        }
      }
      for (int i = threadIdx.x; i < n; i += blockDim.x) G.u[i] += (double)Ls[0].u[i];
      __syncthreads();
      ++outer;
    }
    outer_total += outer;
    if (isnan(resid)) { status = RICH_ENAN; break; }
    // history shift
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      psinm1[i] = psin[i];
      psin[i] = G.u[i];
      if (fresh) thn[i] = thcur[i];
    }
    __syncthreads();
    have_prev = 1;
  }
  if (threadIdx.x == 0) {
    A.have_prev[c] = have_prev;
    A.thn_valid[c] = th_valid;
    A.st_status[c] = status;
    A.st_cycles[c] = cyc_total;
    A.st_outer[c] = outer_total;
    A.st_resid[c] = resid;
    A.st_updates[c] = updates;
  }
  __syncthreads();
}

template <int MODEL>
__global__ void __launch_bounds__(COL_THREADS_MAX, 1) k_columns(ColArgs A) {
  extern __shared__ float smem[];
  __shared__ Level<float> Ls[COL_MAXLEV];
  __shared__ unsigned long long sm[33];
  __shared__ double kb64[2];
  __shared__ int s_col, s_nl;
  for (;;) {
    if (threadIdx.x == 0) {
      const int k = A.begin + atomicAdd(A.queue, 1);
      s_col = k < A.end ? A.order[k] : -1;
    }
    __syncthreads();
    const int c = s_col;
    __syncthreads();
    if (c < 0) break;
    column_solve<MODEL>(A, c, smem, Ls, &s_nl, kb64, sm);
  }
}

// shared memory of one column of n cells
size_t column_smem(int n, int coarsest_max_n) {
  size_t floats = 0;
  int nn = n, l = 0;
  for (;;) {
    floats += (size_t)COL_ARRAYS * nn + 2;
    ++l;
    if (nn <= coarsest_max_n || l >= COL_MAXLEV) break;
    nn = (nn + 1) / 2;
  }
  return floats * sizeof(float);
}

}  // namespace
}  // namespace rich

using rich::ColArgs;
using rich::ColDesc;

// Columns go to three length classes (more than 512 cells, 257-512, at most
// 256), each a persistent launch whose blocks hold the shared memory of the
// class's longest column and take threads, threads/2, threads/4 (at least
// 32): short columns then fit several blocks per SM.  The classes run
// concurrently (the two shorter ones on streams of their own, ordered by
// events); a column's arithmetic does not depend on its block's size (its
// only reductions are maxima), so the results are those of any one launch.
constexpr int COL_CLASSES = 3;
inline int column_class(int n) { return n > 512 ? 0 : (n > 256 ? 1 : 2); }

struct richards_columns {
  cudaStream_t s = nullptr;
  int ncol = 0, max_n = 0, model = 0, threads = 256;
  int cls_begin[COL_CLASSES] = {0, 0, 0}, cls_end[COL_CLASSES] = {0, 0, 0}, cls_maxn[COL_CLASSES] = {0, 0, 0};
  cudaStream_t aux[COL_CLASSES - 1] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[COL_CLASSES - 1] = {nullptr, nullptr};
  long long ncell = 0;
  richards_opts opts{};
  richards_sink sink{};
  std::vector<ColDesc> host_cols;
  ColDesc* cols = nullptr;
  int *order = nullptr, *queue = nullptr, *thn_valid = nullptr, *have_prev = nullptr;
  double *psin = nullptr, *psinm1 = nullptr, *u = nullptr, *g = nullptr, *Kc = nullptr, *thn = nullptr,
         *thcur = nullptr, *smax = nullptr;
  int *st_status = nullptr, *st_cycles = nullptr, *st_outer = nullptr;
  double* st_resid = nullptr;
  unsigned long long* st_updates = nullptr;
  std::vector<void*> allocs;
  bool have_state = false;
};

namespace {

template <typename T>
bool col_alloc(richards_columns* c, T** p, long long n) {
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * (size_t)(n > 0 ? n : 1)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->allocs.push_back(q);
  *p = (T*)q;
  return true;
}

richards_status launch_columns(richards_columns* c, double dt, int nsteps, int scheme, int threads) {
  using namespace rich;
  ColArgs A{};
  A.cols = c->cols; A.order = c->order; A.ncol = c->ncol; A.queue = c->queue; A.thn_valid = c->thn_valid;
  A.psin = c->psin; A.psinm1 = c->psinm1; A.u = c->u; A.g = c->g; A.Kc = c->Kc; A.thn = c->thn;
  A.thcur = c->thcur; A.smax = c->smax; A.have_prev = c->have_prev;
  A.st_status = c->st_status; A.st_cycles = c->st_cycles; A.st_outer = c->st_outer; A.st_resid = c->st_resid;
  A.st_updates = c->st_updates;
  const richards_opts& o = c->opts;
  A.sink = c->sink.enabled;
  A.h1 = c->sink.h1; A.h2 = c->sink.h2; A.h3 = c->sink.h3; A.h4 = c->sink.h4;
  A.xi = o.xi; A.kappa = o.kappa_mode == 0 ? o.kappa : 0.0; A.tol = o.tol; A.inner_rtol = o.inner_rtol;
  A.crtol = o.coarse_rtol; A.dt = dt; A.newton_k = o.newton_iters; A.max_outer = o.max_outer;
  A.inner_cycles = o.inner_cycles; A.nu1 = o.nu1; A.nu2 = o.nu2; A.cmax = o.coarse_max_sweeps;
  A.gamma = o.cycle_gamma; A.gamma_levels = o.gamma_levels; A.coarsest_max_n = o.coarsest_max_n;
  A.scheme = scheme; A.nsteps = nsteps; A.model = c->model; A.lag = o.bdf2_lag;
  A.fp64 = o.precision == 2 ? 1 : 0;
  auto kern = c->model == HAVERKAMP ? k_columns<HAVERKAMP> : (c->model == GARDNER ? k_columns<GARDNER>
                                                                                  : k_columns<VANGENUCHTEN>);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)column_smem(c->max_n, o.coarsest_max_n)) != cudaSuccess)
    return RICH_EINVAL;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMemsetAsync(c->queue, 0, sizeof(int) * COL_CLASSES, c->s) != cudaSuccess) return RICH_ECUDA;
  if (cudaEventRecord(c->ev_fork, c->s) != cudaSuccess) return RICH_ECUDA;
  for (int k = 0; k < COL_CLASSES; ++k) {
    const int count = c->cls_end[k] - c->cls_begin[k];
    if (count <= 0) continue;
    cudaStream_t s = k == 0 ? c->s : c->aux[k - 1];
    if (k > 0 && cudaStreamWaitEvent(s, c->ev_fork, 0) != cudaSuccess) return RICH_ECUDA;
    const int t = std::max(32, threads >> k);
    const size_t smem = column_smem(c->cls_maxn[k], o.coarsest_max_n);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, t, smem) != cudaSuccess || per_sm < 1)
      return RICH_EINVAL;
    ColArgs Ak = A;
    Ak.begin = c->cls_begin[k];
    Ak.end = c->cls_end[k];
    Ak.queue = c->queue + k;
    kern<<<std::min(nsm * per_sm, count), t, smem, s>>>(Ak);
    if (cudaGetLastError() != cudaSuccess) return RICH_ECUDA;
    if (k > 0 && (cudaEventRecord(c->ev_join[k - 1], s) != cudaSuccess ||
                  cudaStreamWaitEvent(c->s, c->ev_join[k - 1], 0) != cudaSuccess))
      return RICH_ECUDA;
  }
  if (cudaStreamSynchronize(c->s) != cudaSuccess) return RICH_ECUDA;
  return RICH_OK;
}

}  // namespace

extern "C" {

richards_status richards_columns_create(int ncol, const richards_column* cols, const richards_sink* sink,
                                        const richards_opts* opts, void* stream, richards_columns** out) {
  if (!out) return RICH_EINVAL;
  *out = nullptr;
  if (ncol < 1 || !cols || !sink || !opts) return RICH_EINVAL;
  const richards_opts& o = *opts;
  if (o.nu1 < 0 || o.nu2 < 0 || o.coarse_max_sweeps < 1 || o.coarsest_max_n < 1 || !(o.tol > 0.0) ||
      o.newton_iters < 0 || o.newton_iters > 200 || (o.kappa_mode != 0 && o.kappa_mode != 2) || o.ordering != 1 ||
      !(o.xi >= 0.0) || !(o.kappa >= 0.0) || o.inner_cycles < 1 || o.max_outer < 0 || o.cycle_gamma < 1 ||
      o.cycle_gamma > 3 || o.gamma_levels < 0 || o.precision < 0 || o.precision > 2 ||
      (o.bdf2_lag != 0 && o.bdf2_lag != 1))
    return RICH_EINVAL;
  if (rich::sink_error(*sink)) return RICH_EINVAL;
  const int model = cols[0].soil.model;
  std::vector<ColDesc> hc(ncol);
  long long off = 0;
  int max_n = 0;
  for (int k = 0; k < ncol; ++k) {
    const richards_column& q = cols[k];
    const richards_soil& s = q.soil;
    if (q.n < 1 || q.n > RICHARDS_COLUMN_MAX_CELLS || !(q.L > 0.0) || s.model != model) return RICH_EINVAL;
    if (rich::law_error(s.model, s.Ks, s.theta_s, s.theta_r, s.p1, s.p2, s.p3, s.p4, false, false))
      return RICH_EINVAL;
    for (int f = 0; f < 2; ++f) {
      if (q.bc_kind[f] < 0 || q.bc_kind[f] > 3 || !std::isfinite(q.bc_value[f])) return RICH_EINVAL;
      if (q.bc_kind[f] == RICH_BC_FREE_DRAINAGE && f != 0) return RICH_EINVAL;
    }
    ColDesc& d = hc[k];
    d.off = off;
    d.n = q.n;
    d.bc_kind[0] = q.bc_kind[0]; d.bc_kind[1] = q.bc_kind[1];
    d.bc_val[0] = q.bc_value[0]; d.bc_val[1] = q.bc_value[1];
    d.Lz = q.L; d.Ks = s.Ks; d.ts = s.theta_s; d.tr = s.theta_r;
    d.p1 = s.p1; d.p2 = s.p2; d.p3 = s.p3; d.p4 = s.p4;
    off += q.n;
    max_n = std::max(max_n, q.n);
  }
  richards_columns* c = new richards_columns();
  c->s = (cudaStream_t)stream;
  c->ncol = ncol;
  c->max_n = max_n;
  c->model = model;
  c->ncell = off;
  c->opts = o;
  c->sink = *sink;
  c->host_cols = hc;
  // longest first: a greedy queue then balances the blocks
  std::vector<int> order(ncol);
  for (int k = 0; k < ncol; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hc[a].n > hc[b].n; });
  for (int q = 0; q < ncol; ++q) {               // (longest first: each class is one range of order)
    const int k = column_class(hc[order[q]].n);
    if (c->cls_end[k] == c->cls_begin[k]) {
      c->cls_begin[k] = q;
      c->cls_maxn[k] = hc[order[q]].n;
    }
    c->cls_end[k] = q + 1;
  }
  const long long N = off;
  bool ok = col_alloc(c, &c->cols, ncol) && col_alloc(c, &c->order, ncol) &&
            col_alloc(c, &c->queue, COL_CLASSES) &&
            col_alloc(c, &c->thn_valid, ncol) && col_alloc(c, &c->have_prev, ncol) && col_alloc(c, &c->psin, N) &&
            col_alloc(c, &c->psinm1, N) && col_alloc(c, &c->u, N) && col_alloc(c, &c->g, N) &&
            col_alloc(c, &c->Kc, N) && col_alloc(c, &c->thn, N) && col_alloc(c, &c->thcur, N) &&
            col_alloc(c, &c->smax, N) && col_alloc(c, &c->st_status, ncol) && col_alloc(c, &c->st_cycles, ncol) &&
            col_alloc(c, &c->st_outer, ncol) && col_alloc(c, &c->st_resid, ncol) &&
            col_alloc(c, &c->st_updates, ncol);
  for (int k = 0; ok && k < COL_CLASSES - 1; ++k)
    ok = cudaStreamCreateWithFlags(&c->aux[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    richards_columns_destroy(c);
    return RICH_ENOMEM;
  }
  // sink coefficient of every cell (same reading as richards_set_sink)
  std::vector<double> smax(N, 0.0);
  if (sink->enabled) {
    const double lam = sink->root_decay, D = sink->root_depth;
    const double Z = lam * (1.0 - std::exp(-D / lam));
    for (int k = 0; k < ncol; ++k) {
      const int nk = hc[k].n;
      for (int i = 0; i < nk; ++i) {
        const double depth = hc[k].Lz * (double)(2 * (nk - 1 - i) + 1) / (double)(2 * nk);
        smax[hc[k].off + i] = depth <= D ? sink->Tp * std::exp(-depth / lam) / Z : 0.0;
      }
    }
  }
  if (cudaMemcpy(c->cols, hc.data(), sizeof(ColDesc) * ncol, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->order, order.data(), sizeof(int) * ncol, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->smax, smax.data(), sizeof(double) * N, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->thn_valid, 0, sizeof(int) * ncol) != cudaSuccess ||
      cudaMemset(c->have_prev, 0, sizeof(int) * ncol) != cudaSuccess) {
    richards_columns_destroy(c);
    return RICH_ECUDA;
  }
  // shared memory of the longest column must fit one block
  const size_t smem = rich::column_smem(max_n, o.coarsest_max_n);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if ((long long)smem + 4096 > optin) {
    richards_columns_destroy(c);
    return RICH_EINVAL;
  }
  *out = c;
  return RICH_OK;
}

void richards_columns_destroy(richards_columns* c) {
  if (!c) return;
  if (c->s) cudaStreamSynchronize(c->s); else cudaDeviceSynchronize();
  for (int k = 0; k < COL_CLASSES - 1; ++k) {
    if (c->aux[k]) { cudaStreamSynchronize(c->aux[k]); cudaStreamDestroy(c->aux[k]); }
    if (c->ev_join[k]) cudaEventDestroy(c->ev_join[k]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (void* p : c->allocs) cudaFree(p);
  delete c;
}

long long richards_columns_ncell(const richards_columns* c) { return c ? c->ncell : 0; }

richards_status richards_columns_set_state(richards_columns* c, const double* psi, const double* psi_prev) {
  if (!c || !psi) return RICH_EINVAL;
  const long long N = c->ncell;
  for (long long i = 0; i < N; ++i)
    if (!std::isfinite(psi[i]) || (psi_prev && !std::isfinite(psi_prev[i]))) return RICH_EINVAL;
  if (cudaMemcpyAsync(c->psin, psi, sizeof(double) * N, cudaMemcpyHostToDevice, c->s) != cudaSuccess)
    return RICH_ECUDA;
  if (psi_prev &&
      cudaMemcpyAsync(c->psinm1, psi_prev, sizeof(double) * N, cudaMemcpyHostToDevice, c->s) != cudaSuccess)
    return RICH_ECUDA;
  std::vector<int> hp(c->ncol, psi_prev ? 1 : 0);
  if (cudaMemcpyAsync(c->have_prev, hp.data(), sizeof(int) * c->ncol, cudaMemcpyHostToDevice, c->s) != cudaSuccess ||
      cudaMemsetAsync(c->thn_valid, 0, sizeof(int) * c->ncol, c->s) != cudaSuccess ||
      cudaStreamSynchronize(c->s) != cudaSuccess)
    return RICH_ECUDA;
  c->have_state = true;
  return RICH_OK;
}

richards_status richards_columns_run(richards_columns* c, double dt, int nsteps, int scheme) {
  if (!c || !c->have_state || !(dt > 0.0) || !std::isfinite(dt) || nsteps < 0 || (scheme != 1 && scheme != 2))
    return RICH_EINVAL;
  if (nsteps == 0) return RICH_OK;
  return launch_columns(c, dt, nsteps, scheme, c->threads);
}

richards_status richards_columns_get_state(richards_columns* c, double* psi, int on_device) {
  if (!c || !psi || !c->have_state) return RICH_EINVAL;
  if (cudaMemcpyAsync(psi, c->psin, sizeof(double) * c->ncell,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->s) != cudaSuccess ||
      cudaStreamSynchronize(c->s) != cudaSuccess)
    return RICH_ECUDA;
  return RICH_OK;
}

richards_status richards_columns_stats(richards_columns* c, int* status, int* cycles, int* outer, double* resid,
                                       long long* updates) {
  if (!c) return RICH_EINVAL;
  const int n = c->ncol;
  std::vector<unsigned long long> up(n);
  if ((status && cudaMemcpy(status, c->st_status, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (cycles && cudaMemcpy(cycles, c->st_cycles, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (outer && cudaMemcpy(outer, c->st_outer, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (resid && cudaMemcpy(resid, c->st_resid, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (updates && cudaMemcpy(up.data(), c->st_updates, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost) !=
                      cudaSuccess))
    return RICH_ECUDA;
  if (updates)
    for (int k = 0; k < n; ++k) updates[k] = (long long)up[k];
  return RICH_OK;
}

richards_status richards_columns_set_threads(richards_columns* c, int threads) {
  if (!c || (threads != 64 && threads != 128 && threads != 256 && threads != 512)) return RICH_EINVAL;
  c->threads = threads;
  return RICH_OK;
}

richards_status richards_columns_autotune(richards_columns* c, double dt, int scheme, int* threads_out) {
  if (!c || !c->have_state) return RICH_EINVAL;
  // each candidate runs one untimed step and then two timed steps, each run
  // from the current state on the same data; the state is restored afterwards
  const long long N = c->ncell;
  std::vector<double> psin(N), psinm1(N);
  std::vector<int> hp(c->ncol), tv(c->ncol);
  if (cudaMemcpy(psin.data(), c->psin, sizeof(double) * N, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(psinm1.data(), c->psinm1, sizeof(double) * N, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hp.data(), c->have_prev, sizeof(int) * c->ncol, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(tv.data(), c->thn_valid, sizeof(int) * c->ncol, cudaMemcpyDeviceToHost) != cudaSuccess)
    return RICH_ECUDA;
  const int cand[] = {128, 256, 512};
  float best = 1e30f;
  int best_t = c->threads;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto restore = [&]() {
    return cudaMemcpy(c->psin, psin.data(), sizeof(double) * N, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(c->psinm1, psinm1.data(), sizeof(double) * N, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(c->have_prev, hp.data(), sizeof(int) * c->ncol, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(c->thn_valid, tv.data(), sizeof(int) * c->ncol, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  for (int t : cand) {
    if (!restore()) return RICH_ECUDA;
    if (launch_columns(c, dt, 1, scheme, t) != RICH_OK) continue;
    if (!restore()) return RICH_ECUDA;
    cudaEventRecord(e0, c->s);
    const richards_status st = launch_columns(c, dt, 2, scheme, t);
    cudaEventRecord(e1, c->s);
    cudaEventSynchronize(e1);
    if (st != RICH_OK) continue;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_t = t; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!restore()) return RICH_ECUDA;
  c->threads = best_t;
  if (threads_out) *threads_out = best_t;
  return RICH_OK;
}

}  // extern "C"
