/*
 * CPU FP64 oracle for the NGS-FAS Richards solver -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential implementation of what the method computes, used
 * to check the CUDA path.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does.  It shares no
 * code, header or table with the CUDA library.
 *
 * What it follows (paper sections / equations):
 *   - constitutive laws theta(psi), K(psi): Table 1 (Haverkamp, Mualem-van
 *     Genuchten with l = 0.5, Gardner), saturated branch psi >= 0 -> theta_s, K_s;
 *   - face-averaged conductivity and the conservative finite-difference
 *     operator: Section 2, eq. (discrete-strong), matrix M of Section 2;
 *   - BDF1 with stabilisation xi: eq. (fully-bdf1); BDF2 is not written in the
 *     paper (reading: a = 3/(2 tau), history (4 theta^n - theta^{n-1})/(2 tau),
 *     lagged state 2 psi^n - psi^{n-1});
 *   - NGS with shifted splitting M = L + D_kappa + U_kappa: eq. (iterative) and
 *     the scalar point update eq. (point-update), solved by safeguarded Newton;
 *   - the nonlinear operator N_h and right side g_h: eq. (Nh-def);
 *   - two-grid FAS steps 1-7 and its recursive V-cycle: Section 3.2.
 *
 * Parity status per function is listed in the test suite and in the design
 * notes: the Feddes sink, the BDF2 form, the coarse-grid operators and the
 * odd-size transfers are build-defined readings ("parity unpinned" against the
 * paper; pinned only by self-consistency, mass balance and the FAS fixed point).
 */
#ifndef RICHARDS_ORACLE_H
#define RICHARDS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_HAVERKAMP = 0, ORC_GARDNER = 1, ORC_VANGENUCHTEN = 2 };
enum { ORC_DIRICHLET = 0, ORC_NOFLUX = 1, ORC_FLUX = 2, ORC_FREE_DRAINAGE = 3 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOCONV = 3, ORC_ENAN = 4 };

typedef struct {
  int dim;          /* 1..3; the vertical axis is dim-1 */
  int n[3];         /* cells per axis, n = 1 on unused axes */
  double L[3];      /* lengths */
} orc_grid;

typedef struct {
  int model;
  double Ks, theta_s, theta_r, p1, p2, p3, p4;
  const double *Ks_field, *p1_field, *p2_field;   /* nullable, per cell */
} orc_soil;

/* A material of a layered soil (spatially varying law, Section 4.1's
   composite column and Section 4.2's two-layer field). */
#define ORC_MAXMAT 8
typedef struct {
  int model;
  double Ks, theta_s, theta_r, p1, p2, p3, p4;
} orc_material;

typedef struct {
  int kind[6];                        /* face 2*axis+side */
  double value[6];
  const double *value_field[6];       /* nullable, per face cell */
  const unsigned char *mask_field[6]; /* nullable: Dirichlet where mask != 0 */
} orc_bc;

typedef struct {
  int enabled;
  double Tp, root_depth, root_decay, h1, h2, h3, h4;
} orc_sink;

typedef struct {
  int nu1, nu2;
  int coarse_max_sweeps;
  double coarse_rtol;
  int coarsest_max_n, max_levels;
  int kappa_mode;      /* 0 absolute kappa, 1 Remark 3.1 row-sum equalising, 2 zero */
  double kappa, xi;
  double tol;          /* on tau_eff * ||N(psi) - g||_inf */
  int max_cycles;
  int ordering;        /* 0 lexicographic, 1 red-black */
  int newton_iters;    /* 0: to tolerance; k > 0: exactly k safeguarded steps */
  int cycle_gamma;     /* coarse-grid visits per level: 1 V-cycle, 2 W-cycle */
  int gamma_levels;    /* cycle_gamma applies on levels < gamma_levels (0: all) */
  int fmg_cycles;      /* > 0: full multigrid pass first, this many cycles per level */
  int bdf2_lag;        /* BDF2 state of the lagged K and the xi term: 0 psi* = 2 psi^n -
                          psi^(n-1) (second order), 1 psi* = psi^n (the lag of eq.
                          fully-bdf1) */
} orc_opts;

typedef struct {
  int cycles;
  double resid;        /* tau_eff * ||g - N(psi)||_inf at exit */
  double resid0;
} orc_info;

typedef struct orc_ctx orc_ctx;

orc_ctx *orc_create(const orc_grid *g, const orc_soil *s, const orc_bc *b,
                    const orc_sink *k, const orc_opts *o);
void orc_destroy(orc_ctx *c);
int orc_nlevels(const orc_ctx *c);
void orc_level_n(const orc_ctx *c, int lev, int n_out[3]);
long orc_level_ncell(const orc_ctx *c, int lev);
long orc_face_ncell(const orc_ctx *c, int lev, int face);

/* state psi^n (and psi^{n-1} when psi_prev != NULL) */
void orc_set_state(orc_ctx *c, const double *psi, const double *psi_prev);
void orc_get_state(const orc_ctx *c, double *psi);

/* per-step preparation: a, lagged state, Kc, boundary conductances, g (fine),
   coarse Kc / conductances, kappa.  scheme 2 falls back to BDF1 when no
   previous state exists.  Returns the scheme actually used. */
int orc_prepare(orc_ctx *c, double dt, int scheme);
double orc_a(const orc_ctx *c);

/* N_lev(psi) into out (eq. Nh-def), and r = g - N(psi) with its max norm. */
void orc_apply_N(const orc_ctx *c, int lev, const double *psi, double *out);
double orc_residual(const orc_ctx *c, int lev, const double *psi, const double *g, double *r);

/* smoothing.  color = -1: full sweep in the configured ordering; 0/1: only the
   red/black half of a red-black sweep. */
void orc_sweep(orc_ctx *c, int lev, double *psi, const double *g, int color);
void orc_sweep_ordering(orc_ctx *c, int lev, double *psi, const double *g, int ordering);
/* the red-black sweep on nthreads OpenMP threads (<= 0: all); same result as
   orc_sweep_ordering(..., 1); returns the threads used */
int orc_sweep_rb_threads(orc_ctx *c, int lev, double *psi, const double *g, int nthreads);

/* transfers between lev (fine) and lev+1 (coarse) */
void orc_restrict(const orc_ctx *c, int lev, const double *fine, double *coarse);
void orc_prolong_add(const orc_ctx *c, int lev, const double *coarse, double *fine);

/* one V-cycle on the fine level from psi with right side g (fine) */
void orc_vcycle(orc_ctx *c, int lev, double *psi, const double *g);

/* one implicit time step: prepare, cycle to tolerance, shift history. */
int orc_step(orc_ctx *c, double dt, int scheme, orc_info *info);
/* same, but starting from and returning the caller's iterate, without shifting
   the history (for studies of a single implicit solve). */
int orc_solve_current(orc_ctx *c, double *psi, orc_info *info);
/* Layered soil: nmat (1..ORC_MAXMAT) materials and a material index per
   fine cell (host array, copied).  Each cell then takes its material's law
   and parameters (the soil's scalars and fields no longer apply); a coarse
   cell takes the material with the largest restriction weight among its
   fine cells (ties: the lower index).  Returns ORC_OK or ORC_EINVAL. */
int orc_set_materials(orc_ctx *c, const orc_material *mats, int nmat, const unsigned char *index);
/* Material index of every cell of level lev (0 everywhere without materials). */
void orc_level_material(const orc_ctx *c, int lev, unsigned char *out);
/* Full multigrid pass on the prepared step from the iterate psi (level 0):
   fmg_cycles cycles per level, coarsest first. */
void orc_fmg(orc_ctx *c, double *psi);

/* inspection: which = 0 Kc, 1 g, 2 p1, 3 p2, 4 smax, 5 kappa, 6 psi_star,
   7 hist (a * history part of g), 10+face: boundary conductance on a face */
void orc_get_array(const orc_ctx *c, int lev, int which, double *out);
void orc_set_g(orc_ctx *c, const double *g);

/* pointwise constitutive laws with a cell's parameters at a level */
void orc_soil_eval(const orc_ctx *c, int lev, long cell, double psi,
                   double *theta, double *dtheta, double *K);
void orc_sink_eval(const orc_ctx *c, int lev, long cell, double psi, double *S, double *dS);

/* scalar point solve of eq. (point-update): a theta(x) + S(x) + cc x = f */
double orc_point_solve(const orc_ctx *c, int lev, long cell, double cc, double f,
                       double x0, int newton_iters, int *iters_out);

/* dense operator matrix of a level (ncell^2, row-major): the linear part
   M including the Dirichlet boundary diagonal terms. */
void orc_dense_M(const orc_ctx *c, int lev, double *M);

/* net boundary inflow rate (volume per time) of the fine level at psi:
   Dirichlet face fluxes, prescribed fluxes and free drainage. */
double orc_boundary_inflow(const orc_ctx *c, const double *psi);
double orc_cell_volume(const orc_ctx *c, int lev);

#ifdef __cplusplus
}
#endif
#endif
