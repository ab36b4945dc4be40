/*
 * CPU FP64 oracle for the NGS-FAS Richards solver -- TEST INFRASTRUCTURE ONLY.
 * (Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file's library.  It shares nothing with the CUDA path.)
 *
 * Plain, sequential, double precision, built without fast-math and without
 * floating-point contraction.  Every function cites the passage of the paper
 * it follows; build-defined readings are marked "reading".
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include "richards_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXLEV 24
#define MAXW 8

typedef struct { int cnt; int idx[MAXW]; double w[MAXW]; } wrow;

typedef struct {
  int n[3];
  double h[3];
  long ncell;
  double *Kc, *p1, *p2, *smax, *kappa;
  unsigned char *mat;   /* layered soil: material per cell (NULL otherwise) */
  double *kb[6];
  long nface[6];
  double *g, *psi, *psibar, *d, *tmp;
  /* transfers to the next coarser level (lev < nlev-1), per axis */
  wrow *R[3];   /* R[ax][J]: coarse J <- fine (full weighting, normalised) */
  wrow *P[3];   /* P[ax][i]: fine i <- coarse (linear interpolation) */
} level;

struct orc_ctx {
  orc_grid grid;
  orc_soil soil;          /* scalars; fields copied below */
  int nmat;               /* layered soil: materials as soils (scalars only) */
  orc_soil msoil[ORC_MAXMAT];
  orc_bc bc;              /* kinds/values; fields copied below */
  orc_sink sink;
  orc_opts opts;
  int nlev;
  level lev[MAXLEV];
  double *Ks;             /* fine per-cell Ks */
  double *bcval[6];
  unsigned char *bcmask[6];
  double *psi_n, *psi_nm1, *psistar, *hist;
  int have_prev;
  double a, dt;
  int scheme;
};

/* ------------------------------------------------------------------ */
/* indexing                                                            */
/* ------------------------------------------------------------------ */
static long cidx(const level *L, int i0, int i1, int i2) {
  return (long)i0 + (long)L->n[0] * ((long)i1 + (long)L->n[1] * (long)i2);
}
static void cpos(const level *L, long idx, int ii[3]) {
  ii[0] = (int)(idx % L->n[0]);
  ii[1] = (int)((idx / L->n[0]) % L->n[1]);
  ii[2] = (int)(idx / ((long)L->n[0] * L->n[1]));
}
/* face cell index on axis ax: lexicographic over the other axes, first fastest */
static long fidx(const level *L, int ax, const int ii[3]) {
  long r = 0, mul = 1;
  for (int a = 0; a < 3; ++a) {
    if (a == ax) continue;
    r += (long)ii[a] * mul;
    mul *= L->n[a];
  }
  return r;
}

/* ------------------------------------------------------------------ */
/* constitutive laws: Table 1 (Haverkamp, van Genuchten-Mualem with    */
/* pore-connectivity l, Gardner).  Reading for psi >= 0: theta = theta_s, */
/* K = Ks, theta' = 0 (Gardner's explicit saturated branch, applied to  */
/* all three laws).                                                    */
/* ------------------------------------------------------------------ */
/* the law of cell i of a level: its material's, else the soil's */
static const orc_soil *soil_of(const orc_ctx *c, const level *L, long i) {
  return L->mat ? &c->msoil[L->mat[i]] : &c->soil;
}

static void soil_law(const orc_soil *s, double p1, double p2, double Ks, double psi,
                     double *th, double *dth, double *K) {
  const double ts = s->theta_s, tr = s->theta_r;
  if (!(psi < 0.0)) {
    if (th) *th = ts;
    if (dth) *dth = 0.0;
    if (K) *K = Ks;
    return;
  }
  const double h = -psi;   /* suction head |psi| */
  if (s->model == ORC_HAVERKAMP) {
    /* theta = theta_r + alpha (theta_s - theta_r) / (alpha + |psi|^beta)
       K = Ks A / (A + |psi|^gamma)                                     */
    const double alpha = p1, beta = p2, A = s->p3, gam = s->p4;
    const double u = pow(h, beta);
    if (th) *th = tr + alpha * (ts - tr) / (alpha + u);
    if (dth) *dth = alpha * (ts - tr) * beta * pow(h, beta - 1.0) / ((alpha + u) * (alpha + u));
    if (K) *K = Ks * A / (A + pow(h, gam));
  } else if (s->model == ORC_GARDNER) {
    /* theta = theta_r + (theta_s - theta_r) e^{alpha psi},  K = Ks e^{alpha psi} */
    const double alpha = p1;
    const double e = exp(alpha * psi);
    if (th) *th = tr + (ts - tr) * e;
    if (dth) *dth = alpha * (ts - tr) * e;
    if (K) *K = Ks * e;
  } else {
    /* Se = (1 + (alpha |psi|)^n)^{-m}, m = 1 - 1/n
       theta = theta_r + (theta_s - theta_r) Se
       K = Ks Se^l [1 - (1 - Se^{1/m})^m]^2                              */
    const double alpha = p1, n = p2, l = s->p3;
    const double m = 1.0 - 1.0 / n;
    const double t = pow(alpha * h, n);
    const double Se = pow(1.0 + t, -m);
    if (th) *th = tr + (ts - tr) * Se;
    if (dth) *dth = (ts - tr) * m * n * (t / h) * pow(1.0 + t, -m - 1.0);
    if (K) {
      const double inner = 1.0 - pow(1.0 - pow(Se, 1.0 / m), m);
      *K = Ks * pow(Se, l) * inner * inner;
    }
  }
}

/* Reading of the unspecified root-water-uptake sink S(psi): Feddes-type
   S = alpha_F(psi) * smax_cell, alpha_F piecewise linear through
   (h4,0), (h3,1), (h2,1), (h1,0), zero outside; S' is the right derivative.
   On [h4, h3] S' >= 0, the rising branch of assumption (A2). */
static void sink_law(const orc_sink *k, double smax, double psi, double *S, double *dS) {
  double a = 0.0, da = 0.0;
  if (k->enabled && smax > 0.0) {
    if (psi >= k->h1 || psi < k->h4) {
      a = 0.0; da = 0.0;
    } else if (psi >= k->h2) {
      a = (k->h1 - psi) / (k->h1 - k->h2); da = -1.0 / (k->h1 - k->h2);
    } else if (psi >= k->h3) {
      a = 1.0; da = 0.0;
    } else {
      a = (psi - k->h4) / (k->h3 - k->h4); da = 1.0 / (k->h3 - k->h4);
    }
  }
  if (S) *S = a * smax;
  if (dS) *dS = da * smax;
}

static int face_is_dirichlet(const orc_ctx *c, int f, long fc) {
  if (c->bc.kind[f] != ORC_DIRICHLET) return 0;
  if (c->bcmask[f] && !c->bcmask[f][fc]) return 0;
  return 1;
}
static double face_value(const orc_ctx *c, int f, long fc) {
  return c->bcval[f] ? c->bcval[f][fc] : c->bc.value[f];
}

/* ------------------------------------------------------------------ */
/* transfers (Section 3.2: full-weighting restriction, linear          */
/* interpolation).  Reading for cell-centred, possibly non-nested      */
/* levels: N_H = ceil(N/2), H = L/N_H; P interpolates linearly in the  */
/* cell-centre coordinate, with a ghost value equal to the boundary    */
/* cell (constant extrapolation) or, on a fully Dirichlet face, its    */
/* negative (zero correction on the face).  R is the transpose of the  */
/* constant-extrapolation P with every row normalised to sum 1, which  */
/* gives the (1,3,3,1)/8 stencil when the levels are nested.           */
/* ------------------------------------------------------------------ */
static void wrow_add(wrow *r, int j, double w) {
  if (w == 0.0) return;
  for (int k = 0; k < r->cnt; ++k)
    if (r->idx[k] == j) { r->w[k] += w; return; }
  r->idx[r->cnt] = j;
  r->w[r->cnt] = w;
  r->cnt++;
}

static void interp_row(int nf, int nc, int i, double slo, double shi, wrow *row) {
  row->cnt = 0;
  if (nf == 1) { wrow_add(row, 0, 1.0); return; }
  long num = (long)(2 * i + 1) * nc - nf;   /* coarse coordinate = num / (2 nf) */
  long den = 2L * nf;
  long J0 = num >= 0 ? num / den : -((-num + den - 1) / den);
  long rem = num - J0 * den;
  double w = (double)rem / (double)den;
  long J1 = J0 + 1;
  double w0 = 1.0 - w, w1 = w;
  if (J0 < 0) wrow_add(row, 0, w0 * slo); else wrow_add(row, (int)J0, w0);
  if (J1 >= nc) wrow_add(row, nc - 1, w1 * shi); else wrow_add(row, (int)J1, w1);
}

static void build_transfer(const orc_ctx *c, level *F, const level *C) {
  for (int ax = 0; ax < 3; ++ax) {
    int nf = F->n[ax], nc = C->n[ax];
    double slo = 1.0, shi = 1.0;
    if (ax < c->grid.dim) {
      if (c->bc.kind[2 * ax] == ORC_DIRICHLET && !c->bc.mask_field[2 * ax]) slo = -1.0;
      if (c->bc.kind[2 * ax + 1] == ORC_DIRICHLET && !c->bc.mask_field[2 * ax + 1]) shi = -1.0;
    }
    F->P[ax] = (wrow *)calloc((size_t)nf, sizeof(wrow));
    F->R[ax] = (wrow *)calloc((size_t)nc, sizeof(wrow));
    for (int i = 0; i < nf; ++i) interp_row(nf, nc, i, slo, shi, &F->P[ax][i]);
    /* R = normalised transpose of the constant-extrapolation interpolation */
    for (int i = 0; i < nf; ++i) {
      wrow p0;
      interp_row(nf, nc, i, 1.0, 1.0, &p0);
      for (int k = 0; k < p0.cnt; ++k) wrow_add(&F->R[ax][p0.idx[k]], i, p0.w[k]);
    }
    for (int J = 0; J < nc; ++J) {
      double s = 0.0;
      for (int k = 0; k < F->R[ax][J].cnt; ++k) s += F->R[ax][J].w[k];
      for (int k = 0; k < F->R[ax][J].cnt; ++k) F->R[ax][J].w[k] /= s;
    }
  }
}

void orc_restrict(const orc_ctx *c, int lev, const double *fine, double *coarse) {
  const level *F = &c->lev[lev], *C = &c->lev[lev + 1];
  for (int J2 = 0; J2 < C->n[2]; ++J2)
    for (int J1 = 0; J1 < C->n[1]; ++J1)
      for (int J0 = 0; J0 < C->n[0]; ++J0) {
        double s = 0.0;
        const wrow *r0 = &F->R[0][J0], *r1 = &F->R[1][J1], *r2 = &F->R[2][J2];
        for (int a2 = 0; a2 < r2->cnt; ++a2)
          for (int a1 = 0; a1 < r1->cnt; ++a1)
            for (int a0 = 0; a0 < r0->cnt; ++a0)
              s += r0->w[a0] * r1->w[a1] * r2->w[a2] *
                   fine[cidx(F, r0->idx[a0], r1->idx[a1], r2->idx[a2])];
        coarse[cidx(C, J0, J1, J2)] = s;
      }
}

/* restriction of a boundary-face array (the face's two in-plane axes) */
static void restrict_face(const orc_ctx *c, int lev, int ax, const double *fine, double *coarse) {
  const level *F = &c->lev[lev], *C = &c->lev[lev + 1];
  int oa[2], k = 0;
  for (int a = 0; a < 3; ++a) if (a != ax) oa[k++] = a;
  for (int J1 = 0; J1 < C->n[oa[1]]; ++J1)
    for (int J0 = 0; J0 < C->n[oa[0]]; ++J0) {
      const wrow *r0 = &F->R[oa[0]][J0], *r1 = &F->R[oa[1]][J1];
      double s = 0.0;
      for (int a1 = 0; a1 < r1->cnt; ++a1)
        for (int a0 = 0; a0 < r0->cnt; ++a0)
          s += r0->w[a0] * r1->w[a1] * fine[r0->idx[a0] + (long)F->n[oa[0]] * r1->idx[a1]];
      coarse[J0 + (long)C->n[oa[0]] * J1] = s;
    }
}

void orc_prolong_add(const orc_ctx *c, int lev, const double *coarse, double *fine) {
  const level *F = &c->lev[lev], *C = &c->lev[lev + 1];
  for (int i2 = 0; i2 < F->n[2]; ++i2)
    for (int i1 = 0; i1 < F->n[1]; ++i1)
      for (int i0 = 0; i0 < F->n[0]; ++i0) {
        const wrow *p0 = &F->P[0][i0], *p1 = &F->P[1][i1], *p2 = &F->P[2][i2];
        double s = 0.0;
        for (int a2 = 0; a2 < p2->cnt; ++a2)
          for (int a1 = 0; a1 < p1->cnt; ++a1)
            for (int a0 = 0; a0 < p0->cnt; ++a0)
              s += p0->w[a0] * p1->w[a1] * p2->w[a2] *
                   coarse[cidx(C, p0->idx[a0], p1->idx[a1], p2->idx[a2])];
        fine[cidx(F, i0, i1, i2)] += s;
      }
}

/* ------------------------------------------------------------------ */
/* creation                                                            */
/* ------------------------------------------------------------------ */
static double *dalloc(long n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

static void level_alloc(level *L, int dim) {
  L->ncell = (long)L->n[0] * L->n[1] * L->n[2];
  L->Kc = dalloc(L->ncell); L->p1 = dalloc(L->ncell); L->p2 = dalloc(L->ncell);
  L->smax = dalloc(L->ncell); L->kappa = dalloc(L->ncell);
  L->g = dalloc(L->ncell); L->psi = dalloc(L->ncell); L->psibar = dalloc(L->ncell);
  L->d = dalloc(L->ncell); L->tmp = dalloc(L->ncell);
  for (int f = 0; f < 6; ++f) {
    int ax = f / 2;
    if (ax < dim) {
      L->nface[f] = L->ncell / L->n[ax];
      L->kb[f] = dalloc(L->nface[f]);
    } else {
      L->nface[f] = 0;
      L->kb[f] = NULL;
    }
  }
}

orc_ctx *orc_create(const orc_grid *g, const orc_soil *s, const orc_bc *b,
                    const orc_sink *k, const orc_opts *o) {
  if (g->dim < 1 || g->dim > 3) return NULL;
  for (int a = 0; a < 3; ++a) {
    if (g->n[a] < 1) return NULL;
    if (a >= g->dim && g->n[a] != 1) return NULL;
  }
  const int v = g->dim - 1;
  for (int f = 0; f < 2 * g->dim; ++f)
    if (b->kind[f] == ORC_FREE_DRAINAGE && f != 2 * v) return NULL;
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  c->grid = *g; c->soil = *s; c->bc = *b; c->sink = *k; c->opts = *o;
  level *L0 = &c->lev[0];
  for (int a = 0; a < 3; ++a) {
    L0->n[a] = g->n[a];
    L0->h[a] = a < g->dim ? g->L[a] / g->n[a] : 1.0;
  }
  level_alloc(L0, g->dim);
  /* hierarchy: halve every axis with n > 1 until max n <= coarsest_max_n */
  c->nlev = 1;
  for (;;) {
    level *F = &c->lev[c->nlev - 1];
    int mx = 0;
    for (int a = 0; a < 3; ++a) if (F->n[a] > mx) mx = F->n[a];
    if (mx <= o->coarsest_max_n) break;
    if (o->max_levels > 0 && c->nlev >= o->max_levels) break;
    if (c->nlev >= MAXLEV) break;
    level *C = &c->lev[c->nlev];
    for (int a = 0; a < 3; ++a) {
      C->n[a] = F->n[a] > 1 ? (F->n[a] + 1) / 2 : 1;
      C->h[a] = a < g->dim ? g->L[a] / C->n[a] : 1.0;
    }
    level_alloc(C, g->dim);
    c->nlev++;
  }
  const long N = L0->ncell;
  c->Ks = dalloc(N);
  for (long i = 0; i < N; ++i) {
    c->Ks[i] = s->Ks_field ? s->Ks_field[i] : s->Ks;
    L0->p1[i] = s->p1_field ? s->p1_field[i] : s->p1;
    L0->p2[i] = s->p2_field ? s->p2_field[i] : s->p2;
  }
  for (int f = 0; f < 6; ++f) {
    c->bcval[f] = NULL; c->bcmask[f] = NULL;
    c->bc.value_field[f] = NULL; c->bc.mask_field[f] = NULL;
    if (f / 2 >= g->dim) continue;
    long nf = L0->nface[f];
    if (b->value_field[f]) {
      c->bcval[f] = dalloc(nf);
      memcpy(c->bcval[f], b->value_field[f], sizeof(double) * (size_t)nf);
    }
    if (b->mask_field[f]) {
      c->bcmask[f] = (unsigned char *)malloc((size_t)nf);
      memcpy(c->bcmask[f], b->mask_field[f], (size_t)nf);
    }
    c->bc.value_field[f] = c->bcval[f];
    c->bc.mask_field[f] = c->bcmask[f];
  }
  c->soil.Ks_field = c->soil.p1_field = c->soil.p2_field = NULL;
  /* sink coefficient smax = Tp * beta(depth), beta = exp(-d/lambda) normalised
     on [0, root_depth] (reading of the unspecified sink) */
  if (k->enabled) {
    const double lam = k->root_decay, D = k->root_depth;
    const double Z = lam * (1.0 - exp(-D / lam));
    for (long i = 0; i < N; ++i) {
      int ii[3]; cpos(L0, i, ii);
      /* depth of the cell centre below the top face, L (2 (n-1-i) + 1) / (2 n):
         one product and one quotient, so every implementation rounds it the
         same way at the edge of the root zone */
      double depth = g->L[v] * (double)(2 * (L0->n[v] - 1 - ii[v]) + 1) / (double)(2 * L0->n[v]);
      L0->smax[i] = depth <= D ? k->Tp * exp(-depth / lam) / Z : 0.0;
    }
  }
  for (int l = 0; l + 1 < c->nlev; ++l) {
    build_transfer(c, &c->lev[l], &c->lev[l + 1]);
    orc_restrict(c, l, c->lev[l].p1, c->lev[l + 1].p1);
    orc_restrict(c, l, c->lev[l].p2, c->lev[l + 1].p2);
    orc_restrict(c, l, c->lev[l].smax, c->lev[l + 1].smax);
  }
  c->psi_n = dalloc(N); c->psi_nm1 = dalloc(N); c->psistar = dalloc(N); c->hist = dalloc(N);
  return c;
}

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  for (int l = 0; l < c->nlev; ++l) {
    level *L = &c->lev[l];
    free(L->Kc); free(L->p1); free(L->p2); free(L->smax); free(L->kappa);
    free(L->g); free(L->psi); free(L->psibar); free(L->d); free(L->tmp);
    free(L->mat);
    for (int f = 0; f < 6; ++f) free(L->kb[f]);
    for (int a = 0; a < 3; ++a) { free(L->R[a]); free(L->P[a]); }
  }
  for (int f = 0; f < 6; ++f) { free(c->bcval[f]); free(c->bcmask[f]); }
  free(c->Ks); free(c->psi_n); free(c->psi_nm1); free(c->psistar); free(c->hist);
  free(c);
}

/* Layered soil (reading for the coarse levels: the material of largest
   total restriction weight among a coarse cell's fine cells, ties to the
   lower index; every cell uses its material's law and parameters). */
int orc_set_materials(orc_ctx *c, const orc_material *mats, int nmat, const unsigned char *index) {
  if (nmat < 1 || nmat > ORC_MAXMAT || !mats || !index) return ORC_EINVAL;
  level *L0 = &c->lev[0];
  for (long i = 0; i < L0->ncell; ++i)
    if (index[i] >= nmat) return ORC_EINVAL;
  c->nmat = nmat;
  for (int m = 0; m < nmat; ++m) {
    orc_soil *S = &c->msoil[m];
    memset(S, 0, sizeof(*S));
    S->model = mats[m].model;
    S->Ks = mats[m].Ks; S->theta_s = mats[m].theta_s; S->theta_r = mats[m].theta_r;
    S->p1 = mats[m].p1; S->p2 = mats[m].p2; S->p3 = mats[m].p3; S->p4 = mats[m].p4;
  }
  for (int l = 0; l < c->nlev; ++l) {
    level *L = &c->lev[l];
    free(L->mat);
    L->mat = (unsigned char *)malloc((size_t)L->ncell);
  }
  memcpy(L0->mat, index, (size_t)L0->ncell);
  for (int l = 0; l + 1 < c->nlev; ++l) {
    const level *F = &c->lev[l];
    level *C = &c->lev[l + 1];
    for (long J = 0; J < C->ncell; ++J) {
      int jj[3]; cpos(C, J, jj);
      double w[ORC_MAXMAT] = {0};
      const wrow *r0 = &F->R[0][jj[0]], *r1 = &F->R[1][jj[1]], *r2 = &F->R[2][jj[2]];
      for (int a2 = 0; a2 < r2->cnt; ++a2)
        for (int a1 = 0; a1 < r1->cnt; ++a1)
          for (int a0 = 0; a0 < r0->cnt; ++a0) {
            long i = cidx(F, r0->idx[a0], r1->idx[a1], r2->idx[a2]);
            w[F->mat[i]] += r0->w[a0] * r1->w[a1] * r2->w[a2];
          }
      int best = 0;
      for (int m = 1; m < nmat; ++m)
        if (w[m] > w[best]) best = m;
      C->mat[J] = (unsigned char)best;
    }
  }
  for (int l = 0; l < c->nlev; ++l) {
    level *L = &c->lev[l];
    for (long i = 0; i < L->ncell; ++i) {
      const orc_soil *S = &c->msoil[L->mat[i]];
      L->p1[i] = S->p1;
      L->p2[i] = S->p2;
      if (l == 0) c->Ks[i] = S->Ks;
    }
  }
  return ORC_OK;
}

void orc_level_material(const orc_ctx *c, int lev, unsigned char *out) {
  const level *L = &c->lev[lev];
  for (long i = 0; i < L->ncell; ++i) out[i] = L->mat ? L->mat[i] : 0;
}

int orc_nlevels(const orc_ctx *c) { return c->nlev; }
void orc_level_n(const orc_ctx *c, int lev, int n_out[3]) {
  for (int a = 0; a < 3; ++a) n_out[a] = c->lev[lev].n[a];
}
long orc_level_ncell(const orc_ctx *c, int lev) { return c->lev[lev].ncell; }
long orc_face_ncell(const orc_ctx *c, int lev, int face) { return c->lev[lev].nface[face]; }
double orc_a(const orc_ctx *c) { return c->a; }
double orc_cell_volume(const orc_ctx *c, int lev) {
  double V = 1.0;
  for (int a = 0; a < c->grid.dim; ++a) V *= c->lev[lev].h[a];
  return V;
}

void orc_set_state(orc_ctx *c, const double *psi, const double *psi_prev) {
  const long N = c->lev[0].ncell;
  memcpy(c->psi_n, psi, sizeof(double) * (size_t)N);
  if (psi_prev) {
    memcpy(c->psi_nm1, psi_prev, sizeof(double) * (size_t)N);
    c->have_prev = 1;
  } else {
    c->have_prev = 0;
  }
}
void orc_get_state(const orc_ctx *c, double *psi) {
  memcpy(psi, c->psi_n, sizeof(double) * (size_t)c->lev[0].ncell);
}

/* ------------------------------------------------------------------ */
/* operator pieces (Section 2)                                         */
/* ------------------------------------------------------------------ */
/* interior-face coefficient m_f = K_f / h^2, K_f = (Kc_i + Kc_j)/2 (face
   average of the lagged conductivity; the paper's K(psi_{i+e/2}) is read as
   K(psi_{i+e})). */
static double mface(const level *L, long i, long j, int ax) {
  return 0.5 * (L->Kc[i] + L->Kc[j]) / (L->h[ax] * L->h[ax]);
}

/* diagonal m_ii and sum_j m_ij psi_j for cell i */
static void stencil(const orc_ctx *c, const level *L, long i, const double *psi,
                    double *mii, double *offsum) {
  int ii[3]; cpos(L, i, ii);
  double diag = 0.0, off = 0.0;
  for (int ax = 0; ax < c->grid.dim; ++ax) {
    for (int side = 0; side < 2; ++side) {
      int jj[3] = {ii[0], ii[1], ii[2]};
      jj[ax] += side ? 1 : -1;
      if (jj[ax] >= 0 && jj[ax] < L->n[ax]) {
        long j = cidx(L, jj[0], jj[1], jj[2]);
        double m = mface(L, i, j, ax);
        diag += m;
        off += m * psi[j];
      } else {
        /* boundary face: Dirichlet conductance kb over half a cell (reading) */
        long fc = fidx(L, ax, ii);
        diag += 2.0 * L->kb[2 * ax + side][fc] / (L->h[ax] * L->h[ax]);
      }
    }
  }
  *mii = diag;
  *offsum = off;
}

/* N_h(psi) = a theta(psi) + S(psi) + xi psi + M(psi^n) psi   (eq. Nh-def) */
void orc_apply_N(const orc_ctx *c, int lev, const double *psi, double *out) {
  const level *L = &c->lev[lev];
  for (long i = 0; i < L->ncell; ++i) {
    double th, S, mii, off;
    soil_law(soil_of(c, L, i), L->p1[i], L->p2[i], 0.0, psi[i], &th, NULL, NULL);
    sink_law(&c->sink, L->smax[i], psi[i], &S, NULL);
    stencil(c, L, i, psi, &mii, &off);
    out[i] = c->a * th + S + c->opts.xi * psi[i] + mii * psi[i] - off;
  }
}

double orc_residual(const orc_ctx *c, int lev, const double *psi, const double *g, double *r) {
  const level *L = &c->lev[lev];
  double *Np = dalloc(L->ncell);
  orc_apply_N(c, lev, psi, Np);
  double mx = 0.0;
  for (long i = 0; i < L->ncell; ++i) {
    double ri = g[i] - Np[i];
    if (r) r[i] = ri;
    if (isnan(ri)) mx = NAN;
    else if (fabs(ri) > mx) mx = fabs(ri);
  }
  free(Np);
  return mx;
}

/* kappa per cell (Lemma 3.1 splitting shift).  Mode 0: absolute value;
   mode 1: Remark 3.1, kappa_i = max_k u_k - u_i with u_i the row sum of the
   strictly upper part for the current ordering; mode 2: zero. */
static void compute_kappa(orc_ctx *c, level *L) {
  if (c->opts.kappa_mode != 1) {
    double k = c->opts.kappa_mode == 0 ? c->opts.kappa : 0.0;
    for (long i = 0; i < L->ncell; ++i) L->kappa[i] = k;
    return;
  }
  double umax = 0.0;
  for (long i = 0; i < L->ncell; ++i) {
    int ii[3]; cpos(L, i, ii);
    int color = (ii[0] + ii[1] + ii[2]) & 1;
    double u = 0.0;
    for (int ax = 0; ax < c->grid.dim; ++ax)
      for (int side = 0; side < 2; ++side) {
        int jj[3] = {ii[0], ii[1], ii[2]};
        jj[ax] += side ? 1 : -1;
        if (jj[ax] < 0 || jj[ax] >= L->n[ax]) continue;
        long j = cidx(L, jj[0], jj[1], jj[2]);
        int later = c->opts.ordering == 0 ? (j > i) : (color == 0);
        if (later) u += mface(L, i, j, ax);
      }
    L->kappa[i] = u;
    if (u > umax) umax = u;
  }
  for (long i = 0; i < L->ncell; ++i) L->kappa[i] = umax - L->kappa[i];
}

/* Per-step set-up: eq. (fully-bdf1) for BDF1; BDF2 is a reading (see header).
   g_h = a*history + xi psi* - M(psi*) z + boundary terms (eq. Nh-def with the
   known boundary data moved to the right side). */
int orc_prepare(orc_ctx *c, double dt, int scheme) {
  level *L = &c->lev[0];
  const long N = L->ncell;
  const int v = c->grid.dim - 1;
  if (scheme == 2 && !c->have_prev) scheme = 1;
  c->scheme = scheme;
  c->dt = dt;
  c->a = scheme == 1 ? 1.0 / dt : 1.5 / dt;
  for (long i = 0; i < N; ++i) {
    double thn, thm = 0.0;
    soil_law(soil_of(c, L, i), L->p1[i], L->p2[i], c->Ks[i], c->psi_n[i], &thn, NULL, NULL);
    if (scheme == 1) {
      c->psistar[i] = c->psi_n[i];
      c->hist[i] = thn / dt;
    } else {
      soil_law(soil_of(c, L, i), L->p1[i], L->p2[i], c->Ks[i], c->psi_nm1[i], &thm, NULL, NULL);
      c->psistar[i] = c->opts.bdf2_lag ? c->psi_n[i] : 2.0 * c->psi_n[i] - c->psi_nm1[i];
      c->hist[i] = (4.0 * thn - thm) / (2.0 * dt);
    }
    soil_law(soil_of(c, L, i), L->p1[i], L->p2[i], c->Ks[i], c->psistar[i], NULL, NULL, &L->Kc[i]);
  }
  /* boundary face conductances of the fine level */
  for (int f = 0; f < 2 * c->grid.dim; ++f) {
    const int ax = f / 2, side = f % 2;
    for (long i = 0; i < N; ++i) {
      int ii[3]; cpos(L, i, ii);
      if (ii[ax] != (side ? L->n[ax] - 1 : 0)) continue;
      long fc = fidx(L, ax, ii);
      if (face_is_dirichlet(c, f, fc)) {
        double Kb;
        soil_law(soil_of(c, L, i), L->p1[i], L->p2[i], c->Ks[i], face_value(c, f, fc), NULL, NULL, &Kb);
        L->kb[f][fc] = 0.5 * (L->Kc[i] + Kb);
      } else {
        L->kb[f][fc] = 0.0;
      }
    }
  }
  /* right side g */
  for (long i = 0; i < N; ++i) {
    int ii[3]; cpos(L, i, ii);
    double gi = c->hist[i] + c->opts.xi * c->psistar[i];
    /* gravity: -(M z)_i = (K_{i+e_z/2} - K_{i-e_z/2}) / h_z over interior z-faces */
    if (ii[v] + 1 < L->n[v]) {
      int jj[3] = {ii[0], ii[1], ii[2]}; jj[v] += 1;
      gi += 0.5 * (L->Kc[i] + L->Kc[cidx(L, jj[0], jj[1], jj[2])]) / L->h[v];
    }
    if (ii[v] > 0) {
      int jj[3] = {ii[0], ii[1], ii[2]}; jj[v] -= 1;
      gi -= 0.5 * (L->Kc[i] + L->Kc[cidx(L, jj[0], jj[1], jj[2])]) / L->h[v];
    }
    /* boundary faces (reading): Dirichlet m_b (psi_b + z_b - z_i) with
       m_b = 2 K_b / h^2; prescribed inflow q / h; free drainage -Kc / h_z */
    for (int ax = 0; ax < c->grid.dim; ++ax)
      for (int side = 0; side < 2; ++side) {
        if (ii[ax] != (side ? L->n[ax] - 1 : 0)) continue;
        const int f = 2 * ax + side;
        long fc = fidx(L, ax, ii);
        const double h = L->h[ax];
        if (face_is_dirichlet(c, f, fc)) {
          double dz = (ax == v) ? (side ? 0.5 * h : -0.5 * h) : 0.0;
          gi += 2.0 * L->kb[f][fc] / (h * h) * (face_value(c, f, fc) + dz);
        } else if (c->bc.kind[f] == ORC_FLUX) {
          gi += face_value(c, f, fc) / h;
        } else if (c->bc.kind[f] == ORC_FREE_DRAINAGE) {
          gi -= L->Kc[i] / h;
        }
      }
    L->g[i] = gi;
  }
  /* coarse levels (reading: "complete analogy"): restricted Kc and boundary
     conductances; same a, xi, kappa rule */
  for (int l = 0; l + 1 < c->nlev; ++l) {
    orc_restrict(c, l, c->lev[l].Kc, c->lev[l + 1].Kc);
    for (int f = 0; f < 2 * c->grid.dim; ++f)
      restrict_face(c, l, f / 2, c->lev[l].kb[f], c->lev[l + 1].kb[f]);
  }
  for (int l = 0; l < c->nlev; ++l) compute_kappa(c, &c->lev[l]);
  return scheme;
}

void orc_set_g(orc_ctx *c, const double *g) {
  memcpy(c->lev[0].g, g, sizeof(double) * (size_t)c->lev[0].ncell);
}

/* ------------------------------------------------------------------ */
/* scalar point solve of eq. (point-update):                           */
/*   a theta(x) + S(x) + cc x = f,  cc = xi + kappa_i + m_ii > 0        */
/* The left side is strictly increasing, so the root is unique; it     */
/* lies in [(f - a theta_s - smax)/cc, (f - a theta_r)/cc].  Newton from */
/* the previous iterate, bisection whenever a step leaves the bracket  */
/* (the "damped Newton with backtracking" of Section 3.1, read as a    */
/* bracketed Newton method).                                           */
/* ------------------------------------------------------------------ */
static double point_solve(const orc_ctx *c, const level *L, long i, double cc, double f,
                          double x0, int kfixed, int *iters) {
  const double a = c->a;
  const double smax = c->sink.enabled ? L->smax[i] : 0.0;
  if (!(cc > 0.0)) {
    /* a cell with no coupling and no shift (c = 0): add the shift
       kappa (x - x0) with kappa = 1e-6 a, which leaves the root unchanged
       and gives the bracket below */
    const double k = 1e-6 * a;
    f += (k - cc) * x0;
    cc = k;
  }
  const orc_soil *SL = soil_of(c, L, i);
  double lo = (f - a * SL->theta_s - smax) / cc;
  double hi = (f - a * SL->theta_r) / cc;
  double x = x0 < lo ? lo : (x0 > hi ? hi : x0);
  const int maxit = kfixed > 0 ? kfixed : 200;
  int it = 0;
  while (it < maxit) {
    double th, dth, S, dS;
    soil_law(SL, L->p1[i], L->p2[i], 0.0, x, &th, &dth, NULL);
    sink_law(&c->sink, L->smax[i], x, &S, &dS);
    const double F = a * th + S + cc * x - f;
    const double dF = a * dth + dS + cc;
    ++it;
    if (F == 0.0) break;
    if (F > 0.0) hi = x; else lo = x;
    double xn = x - F / dF;
    /* keep a Newton step that lands strictly inside the bracket, or one that
       moves less than round-off (converged); otherwise bisect */
    const double tiny = 1e-15 * (fabs(x) > 1.0 ? fabs(x) : 1.0);
    if (!(xn > lo && xn < hi) && !(fabs(xn - x) <= tiny)) xn = 0.5 * (lo + hi);
    const double step = fabs(xn - x);
    x = xn;
    if (kfixed <= 0 && step <= tiny) break;
  }
  if (iters) *iters = it;
  return x;
}

double orc_point_solve(const orc_ctx *c, int lev, long cell, double cc, double f,
                       double x0, int newton_iters, int *iters_out) {
  return point_solve(c, &c->lev[lev], cell, cc, f, x0, newton_iters, iters_out);
}

/* one point update of eq. (point-update): neighbours enter with their
   current values (new for already-visited cells, old otherwise), the shift
   kappa_i multiplies the cell's old value. */
static void point_update(const orc_ctx *c, const level *L, long i, double *psi, const double *g) {
  double mii, off;
  stencil(c, L, i, psi, &mii, &off);
  const double cc = c->opts.xi + L->kappa[i] + mii;
  const double f = g[i] + off + L->kappa[i] * psi[i];
  psi[i] = point_solve(c, L, i, cc, f, psi[i], c->opts.newton_iters, NULL);
}

/* NGS sweep (eq. iterative).  Lexicographic order s(i) (Section 2, first
   index fastest; Fig. 1) or red-black: colour (i0+i1+i2) mod 2, red first. */
void orc_sweep_ordering(orc_ctx *c, int lev, double *psi, const double *g, int ordering) {
  level *L = &c->lev[lev];
  if (ordering == 0) {
    for (long i = 0; i < L->ncell; ++i) point_update(c, L, i, psi, g);
  } else {
    for (int col = 0; col < 2; ++col)
      for (long i = 0; i < L->ncell; ++i) {
        int ii[3]; cpos(L, i, ii);
        if (((ii[0] + ii[1] + ii[2]) & 1) == col) point_update(c, L, i, psi, g);
      }
  }
}

/* One red-black sweep with the cells of each colour shared among nthreads
   OpenMP threads (nthreads <= 0: all of them).  Cells of one colour do not
   couple -- each reads only cells of the other colour and its own old value
   -- so every cell gets exactly the update of orc_sweep_ordering's
   red-black sweep, whatever the thread count.  Returns the thread count
   used (1 when the library was built without OpenMP).  Used to time the
   oracle on all host cores. */
int orc_sweep_rb_threads(orc_ctx *c, int lev, double *psi, const double *g, int nthreads) {
  level *L = &c->lev[lev];
  int used = 1;
#ifdef _OPENMP
  used = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
  for (int col = 0; col < 2; ++col) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(used)
#endif
    for (long i = 0; i < L->ncell; ++i) {
      int ii[3]; cpos(L, i, ii);
      if (((ii[0] + ii[1] + ii[2]) & 1) == col) point_update(c, L, i, psi, g);
    }
  }
  (void)nthreads;
  return used;
}

void orc_sweep(orc_ctx *c, int lev, double *psi, const double *g, int color) {
  level *L = &c->lev[lev];
  if (color < 0) { orc_sweep_ordering(c, lev, psi, g, c->opts.ordering); return; }
  for (long i = 0; i < L->ncell; ++i) {
    int ii[3]; cpos(L, i, ii);
    if (((ii[0] + ii[1] + ii[2]) & 1) == color) point_update(c, L, i, psi, g);
  }
}

/* coarsest level (reading): NGS sweeps until the defect drops below
   coarse_rtol times its initial value, at most coarse_max_sweeps */
static void coarse_solve(orc_ctx *c, int lev, double *psi, const double *g) {
  double d0 = orc_residual(c, lev, psi, g, NULL);
  for (int s = 0; s < c->opts.coarse_max_sweeps; ++s) {
    orc_sweep(c, lev, psi, g, -1);
    double d = orc_residual(c, lev, psi, g, NULL);
    if (!(d > c->opts.coarse_rtol * d0)) break;
  }
}

/* Two-grid FAS steps 1-7 (Section 3.2) with the coarse solve replaced by a
   recursive call (V-cycle). */
void orc_vcycle(orc_ctx *c, int lev, double *psi, const double *g) {
  if (lev == c->nlev - 1) { coarse_solve(c, lev, psi, g); return; }
  level *F = &c->lev[lev], *C = &c->lev[lev + 1];
  for (int s = 0; s < c->opts.nu1; ++s) orc_sweep(c, lev, psi, g, -1);      /* 1 */
  orc_residual(c, lev, psi, g, F->d);                                       /* 2 */
  orc_restrict(c, lev, psi, C->psibar);                                     /* 3 */
  orc_restrict(c, lev, F->d, C->d);
  orc_apply_N(c, lev + 1, C->psibar, C->g);                                 /* 4 */
  for (long I = 0; I < C->ncell; ++I) { C->g[I] += C->d[I]; C->psi[I] = C->psibar[I]; }
  /* 5: the coarse solve is the recursion itself, done cycle_gamma times
     (1: V-cycle, Section 3.2; 2: W-cycle) */
  int gam = c->opts.cycle_gamma > 1 ? c->opts.cycle_gamma : 1;
  if (c->opts.gamma_levels > 0 && lev >= c->opts.gamma_levels) gam = 1;
  for (int q = 0; q < gam; ++q) orc_vcycle(c, lev + 1, C->psi, C->g);
  for (long I = 0; I < C->ncell; ++I) C->tmp[I] = C->psi[I] - C->psibar[I]; /* 6 */
  orc_prolong_add(c, lev, C->tmp, psi);
  for (int s = 0; s < c->opts.nu2; ++s) orc_sweep(c, lev, psi, g, -1);      /* 7 */
}

/* Full multigrid (Section 3.2: start from the coarsest grid, interpolate the
   solution to successively finer grids, one or several cycles on each).
   Reading: level l solves N_l(psi_l) = g_l with g_{l+1} = R g_l (full
   weighting of the right side) and the coarse operators of the cycle; every
   level starts from the restricted iterate, psi_{l+1} = R psi_l, and the
   interpolation corrects the finer iterate, psi_l += P(psi_{l+1} - R psi_l),
   so that the time step's initial guess is kept on every scale. */
void orc_fmg(orc_ctx *c, double *psi) {
  const int nl = c->nlev;
  if (nl < 2 || c->opts.fmg_cycles <= 0) return;
  for (int l = 0; l + 1 < nl; ++l) {
    level *F = &c->lev[l], *C = &c->lev[l + 1];
    const double *fpsi = l == 0 ? psi : F->psi;
    orc_restrict(c, l, fpsi, C->psibar);
    orc_restrict(c, l, F->g, C->g);
    memcpy(C->psi, C->psibar, sizeof(double) * (size_t)C->ncell);
  }
  for (int k = 0; k < c->opts.fmg_cycles; ++k) orc_vcycle(c, nl - 1, c->lev[nl - 1].psi, c->lev[nl - 1].g);
  for (int l = nl - 2; l >= 0; --l) {
    level *F = &c->lev[l], *C = &c->lev[l + 1];
    double *fpsi = l == 0 ? psi : F->psi;
    for (long I = 0; I < C->ncell; ++I) C->tmp[I] = C->psi[I] - C->psibar[I];
    orc_prolong_add(c, l, C->tmp, fpsi);
    for (int k = 0; k < c->opts.fmg_cycles; ++k) orc_vcycle(c, l, fpsi, F->g);
  }
}

/* cycle until tau_eff ||g - N(psi)||_inf <= tol, tau_eff = 1/a (reading of
   the "prescribed tolerance") */
int orc_solve_current(orc_ctx *c, double *psi, orc_info *info) {
  const double teff = 1.0 / c->a;
  double r = teff * orc_residual(c, 0, psi, c->lev[0].g, NULL);
  int cycles = 0;
  if (info) info->resid0 = r;
  while (!(r <= c->opts.tol) && cycles < c->opts.max_cycles && !isnan(r)) {
    orc_vcycle(c, 0, psi, c->lev[0].g);
    ++cycles;
    r = teff * orc_residual(c, 0, psi, c->lev[0].g, NULL);
  }
  if (info) { info->cycles = cycles; info->resid = r; }
  if (isnan(r)) return ORC_ENAN;
  return r <= c->opts.tol ? ORC_OK : ORC_ENOCONV;
}

int orc_step(orc_ctx *c, double dt, int scheme, orc_info *info) {
  const long N = c->lev[0].ncell;
  orc_prepare(c, dt, scheme);
  double *psi = dalloc(N);
  memcpy(psi, c->psi_n, sizeof(double) * (size_t)N);   /* psi^(0) = psi^n */
  const int fmg = c->nlev > 1 && c->opts.fmg_cycles > 0;
  double r0 = 0.0;
  if (fmg) {                                             /* full multigrid start */
    r0 = orc_residual(c, 0, psi, c->lev[0].g, NULL) / c->a;
    orc_fmg(c, psi);
  }
  int st = orc_solve_current(c, psi, info);
  if (fmg && info) {                                     /* count the pass's finest cycles */
    info->cycles += c->opts.fmg_cycles;
    info->resid0 = r0;
  }
  if (st != ORC_ENAN) {
    memcpy(c->psi_nm1, c->psi_n, sizeof(double) * (size_t)N);
    memcpy(c->psi_n, psi, sizeof(double) * (size_t)N);
    c->have_prev = 1;
  }
  free(psi);
  return st;
}

/* ------------------------------------------------------------------ */
/* inspection                                                          */
/* ------------------------------------------------------------------ */
void orc_get_array(const orc_ctx *c, int lev, int which, double *out) {
  const level *L = &c->lev[lev];
  const double *src = NULL;
  long n = L->ncell;
  switch (which) {
    case 0: src = L->Kc; break;
    case 1: src = L->g; break;
    case 2: src = L->p1; break;
    case 3: src = L->p2; break;
    case 4: src = L->smax; break;
    case 5: src = L->kappa; break;
    case 6: src = c->psistar; n = c->lev[0].ncell; break;
    case 7: src = c->hist; n = c->lev[0].ncell; break;
    default:
      if (which >= 10 && which < 16) { src = L->kb[which - 10]; n = L->nface[which - 10]; }
  }
  if (src) memcpy(out, src, sizeof(double) * (size_t)n);
}

void orc_soil_eval(const orc_ctx *c, int lev, long cell, double psi,
                   double *theta, double *dtheta, double *K) {
  const level *L = &c->lev[lev];
  double Ks = lev == 0 ? c->Ks[cell] : 0.0;
  soil_law(soil_of(c, L, cell), L->p1[cell], L->p2[cell], Ks, psi, theta, dtheta, K);
}

void orc_sink_eval(const orc_ctx *c, int lev, long cell, double psi, double *S, double *dS) {
  sink_law(&c->sink, c->lev[lev].smax[cell], psi, S, dS);
}

void orc_dense_M(const orc_ctx *c, int lev, double *M) {
  const level *L = &c->lev[lev];
  const long N = L->ncell;
  memset(M, 0, sizeof(double) * (size_t)(N * N));
  for (long i = 0; i < N; ++i) {
    int ii[3]; cpos(L, i, ii);
    for (int ax = 0; ax < c->grid.dim; ++ax)
      for (int side = 0; side < 2; ++side) {
        int jj[3] = {ii[0], ii[1], ii[2]};
        jj[ax] += side ? 1 : -1;
        if (jj[ax] >= 0 && jj[ax] < L->n[ax]) {
          long j = cidx(L, jj[0], jj[1], jj[2]);
          double m = mface(L, i, j, ax);
          M[i * N + i] += m;
          M[i * N + j] -= m;
        } else {
          long fc = fidx(L, ax, ii);
          M[i * N + i] += 2.0 * L->kb[2 * ax + side][fc] / (L->h[ax] * L->h[ax]);
        }
      }
  }
}

/* Net inflow through the boundary at psi (fine level): the face fluxes of the
   boundary reading -- Dirichlet K_b ((psi_b + z_b) - (psi_i + z_i)) / (h/2),
   prescribed q, free drainage -Kc -- times the face area. */
double orc_boundary_inflow(const orc_ctx *c, const double *psi) {
  const level *L = &c->lev[0];
  const int v = c->grid.dim - 1;
  const double V = orc_cell_volume(c, 0);
  double Q = 0.0;
  for (long i = 0; i < L->ncell; ++i) {
    int ii[3]; cpos(L, i, ii);
    for (int ax = 0; ax < c->grid.dim; ++ax)
      for (int side = 0; side < 2; ++side) {
        if (ii[ax] != (side ? L->n[ax] - 1 : 0)) continue;
        const int f = 2 * ax + side;
        const long fc = fidx(L, ax, ii);
        const double h = L->h[ax], A = V / h;
        if (face_is_dirichlet(c, f, fc)) {
          double zi = (ii[v] + 0.5) * L->h[v];
          double zb = (ax == v) ? (side ? c->grid.L[v] : 0.0) : zi;
          Q += A * L->kb[f][fc] * ((face_value(c, f, fc) + zb) - (psi[i] + zi)) / (0.5 * h);
        } else if (c->bc.kind[f] == ORC_FLUX) {
          Q += A * face_value(c, f, fc);
        } else if (c->bc.kind[f] == ORC_FREE_DRAINAGE) {
          Q -= A * L->Kc[i];
        }
      }
  }
  return Q;
}
