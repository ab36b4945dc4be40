/*
 * richards.h -- C ABI of the GB300 (sm_103a) NGS-FAS solver for the
 * Richards equation (conservative finite differences, implicit BDF1/BDF2 in
 * time, full-approximation-scheme multigrid with a red-black nonlinear
 * Gauss-Seidel smoother).
 *
 * Every array argument is a plain pointer with an explicit size.  Host input
 * arrays are copied during the call (the caller keeps ownership).  The context
 * owns every device allocation it makes and releases them in
 * richards_destroy().  No exception crosses the ABI: every call returns a
 * richards_status and richards_last_error() holds a message for the last
 * failing call.  A context is bound to one CUDA stream (given at creation;
 * NULL = the legacy default stream) and must not be used from two host
 * threads at once.
 *
 * Layout of every cell array: lexicographic with the first index fastest
 * (Section 2, the flattening s(i)); axis dim-1 is the vertical axis, its
 * low end the bottom (elevation z = 0).  Face arrays (boundary values and
 * masks) are indexed lexicographically over the two other axes.
 *
 * Units are the caller's, used consistently (the paper's 1-d column is in cm
 * and s; SI works the same way).
 */
#ifndef RICHARDS_H
#define RICHARDS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct richards_ctx richards_ctx;   /* opaque; owns its device memory */

typedef enum {
  RICH_OK = 0,
  RICH_EINVAL = 1,    /* invalid argument or parameter                     */
  RICH_ENOMEM = 2,    /* device allocation failed                          */
  RICH_ENOCONV = 3,   /* max_cycles / max_outer reached above tolerance     */
  RICH_ENAN = 4,      /* NaN/Inf in the iterate; state rolled back to psi^n */
  RICH_ETIMEOUT = 5,  /* a bounded device wait gave up                     */
  RICH_ECUDA = 6,     /* a CUDA runtime call failed                        */
  RICH_EBUSY = 7      /* context busy (batch in flight)                    */
} richards_status;

/* Grid (Section 2, reading: cell-centred, h = L/n per axis).  dim in 1..3;
   n[a] >= 1 cells on axis a; axes a >= dim must have n[a] = 1; n[1] and
   n[2] at most 65535 and fewer than 2^31 cells in all. */
typedef struct {
  int dim;
  int n[3];
  double L[3];
} richards_grid;

/* Constitutive laws of Table 1.  Parameters:
     RICH_HAVERKAMP:     p1 = alpha, p2 = beta, p3 = A, p4 = gamma
     RICH_GARDNER:       p1 = alpha
     RICH_VANGENUCHTEN:  p1 = alpha, p2 = n (> 1), p3 = l (Mualem, 0.5)
   Ks_field / p1_field / p2_field: optional per-cell host arrays (ncell
   doubles) replacing the scalar.  For psi >= 0 all laws give theta_s, Ks. */
enum { RICH_HAVERKAMP = 0, RICH_GARDNER = 1, RICH_VANGENUCHTEN = 2 };
typedef struct {
  int model;
  double Ks, theta_s, theta_r, p1, p2, p3, p4;
  const double *Ks_field, *p1_field, *p2_field;
} richards_soil;

/* Boundary conditions per face f = 2*axis + side (side 0 = low end).
     DIRICHLET     value = head psi_b on the face (or value_field per face
                   cell); with mask_field, Dirichlet where mask != 0 and
                   no-flux elsewhere.  Face conductivity (K_i + K(psi_b))/2
                   over half a cell.
     NOFLUX        zero flux (diffusion and gravity).
     FLUX          prescribed inflow rate (volume / area / time) value or
                   value_field.
     FREE_DRAINAGE unit gradient of total head: outflow K(psi*) of the
                   bottom cell; only on the bottom face (axis dim-1, side 0). */
enum { RICH_BC_DIRICHLET = 0, RICH_BC_NOFLUX = 1, RICH_BC_FLUX = 2, RICH_BC_FREE_DRAINAGE = 3 };
typedef struct {
  int kind[6];
  double value[6];
  const double *value_field[6];
  const unsigned char *mask_field[6];
} richards_bc;

/* Root-water-uptake sink S(psi) = alpha_F(psi) Tp beta(depth) (the paper
   leaves S unspecified beyond assumption (A2); this is a Feddes-type reading):
   alpha_F piecewise linear through (h4,0), (h3,1), (h2,1), (h1,0), zero
   outside; beta = exp(-depth/root_decay) normalised on [0, root_depth]. */
typedef struct {
  int enabled;
  double Tp, root_depth, root_decay, h1, h2, h3, h4;
} richards_sink;

/* Solver options.
     nu1, nu2             pre/post NGS sweeps per level (Section 3.2)
     coarse_max_sweeps,   coarsest level: sweeps until the defect drops by
     coarse_rtol          coarse_rtol or coarse_max_sweeps are done
     coarsest_max_n,      coarsen every axis with n > 1 to ceil(n/2) while
     max_levels           max n > coarsest_max_n (max_levels > 0 caps it)
     kappa_mode, kappa    diagonal shift Lambda_kappa of Lemma 3.1: 0 =
                          constant kappa (1/time), 2 = zero
     xi                   stabilisation of eq. (fully-bdf1) (1/time)
     tol                  stop when tau_eff ||N(psi) - g||_inf <= tol,
                          tau_eff = 1/a (residual in theta units)
     max_cycles           V-cycles per step (FP64) / inner cycles (mixed)
     ordering             1 = red-black; 0 = lexicographic, the paper's order
                          (Section 3.1), run hyperplane by hyperplane
                          (i0 + i1 + i2 = const, one launch each): the same
                          iterates as the sequential sweep, for studies and
                          parity, not speed.  Batched columns: 1 only.
     newton_iters         k > 0: exactly k safeguarded Newton steps per point
                          update; 0: to round-off
     precision            0 = FP64 throughout; 1 = FP32 inner cycles on the
                          correction equation inside an outer defect
                          correction whose lagged K, history, defect, water
                          balance and stop test run in float-float
                          arithmetic (laws ~1e-12 relative); 2 = the same
                          FP32 inner cycles inside an FP64 outer defect
                          correction: lagged K, history, right side, the
                          defect that decides the stop test and the water
                          balance in FP64 (float-float defects only steer
                          the corrections in between)
     inner_cycles,        mixed mode: FP32 cycles per outer iteration, stop
     inner_rtol, max_outer  early below max(inner_rtol, 0.3 tol / r) x the
                          initial inner defect (r: the outer defect in theta
                          units); at most max_outer outer iterations
     tail_cells           levels with at most this many cells run in one
                          thread block (the coarse tail of the V-cycle)
     cycle_gamma          coarse-grid visits per level: 1 = V-cycle (the
                          paper's), 2 = W-cycle
     gamma_levels         cycle_gamma applies on the levels above this one
                          (0: on every level); coarser levels use V-cycles
     graphs               1: the FP32 inner solve of the mixed mode as CUDA
                          graphs -- the cycle captured once and replayed,
                          inside a conditional while node that takes the
                          inner stop test on the device (needs a stream
                          other than the legacy default stream and kernel
                          timing off; falls back to direct launches and a
                          host-driven loop otherwise: richards_graph_status) 
     sweep_planes         FP32 half-sweeps: cells per thread along z (1, 2,
                          4 or 8); above 1 a thread loads the operands of
                          its next cell before it solves the current one
     predictor            mixed mode, BDF2 steps: 1 starts the iteration
                          from the extrapolated psi* = 2 psi^n - psi^{n-1}
                          instead of psi^n (same discrete system and stop
                          test; a closer start needs fewer cycles)
     fmg_cycles           > 0: a full multigrid pass (Section 3.2) starts the
                          step (FP64) or each inner solve (mixed): right
                          sides and iterates restricted to every level, the
                          coarsest solved first, each finer iterate corrected
                          by the interpolated coarse change, then fmg_cycles
                          cycles on it; counted in cycles
     layout               mixed modes: 0 = the finest FP32 level of a grid of
                          at least 2^20 cells with an even n0 keeps its
                          per-cell parameters (right side, psi0, soil
                          fields, sink) with each colour's cells packed
                          together, so a half-sweep reads only its own
                          colour's memory; 1 = the natural layout everywhere
                          (same results: only where values sit changes)
     bdf2_lag             BDF2 state at which K and the xi term are lagged:
                          0 = psi* = 2 psi^n - psi^(n-1) (second order in
                          time); 1 = psi* = psi^n, the lag of eq. (fully-bdf1)
                          (first order in the lag, robust where a sharp
                          wetting front makes the extrapolated K jump by
                          orders of magnitude between steps) */
typedef struct {
  int nu1, nu2, coarse_max_sweeps;
  double coarse_rtol;
  int coarsest_max_n, max_levels;
  int kappa_mode;
  double kappa, xi, tol;
  int max_cycles, ordering, newton_iters, precision;
  int inner_cycles;
  double inner_rtol;
  int max_outer, tail_cells, cycle_gamma, gamma_levels, graphs, sweep_planes, predictor, fmg_cycles;
  int layout;
  int bdf2_lag;
} richards_opts;

typedef struct {
  int cycles;            /* V-cycles (FP64) or FP32 inner V-cycles (mixed)  */
  int outer_iters;       /* FP64 defect-correction iterations (mixed)       */
  int scheme_used;       /* 1 or 2 (BDF2 falls back to BDF1 on a first step) */
  double resid0, resid;  /* tau_eff ||g - N(psi)||_inf at start / at exit    */
  long long cell_updates;/* NGS point updates over all levels this step     */
  /* Water balance of the step (conservation, Section 2): tau_eff times
     sum_i V_i (a theta_i - hist_i + S_i + xi (psi_i - psi*_i)) minus the
     net boundary inflow, i.e. the water volume the unconverged residual
     leaves unaccounted (-tau_eff sum_i V_i r_i), summed in FP64 (in
     float-float with precision 1). */
  double mass_defect;
  /* ||N(psi) - g||_inf / min_i (a theta'(psi_i) + S'(psi_i) + xi): bound on
     ||psi - psi_exact||_inf by the diagonal dominance of the Jacobian
     (Lemma 3.1); +inf where that minimum is 0 (saturated cells, xi = 0). */
  double err_bound;
} richards_step_info;

/* Create a context for one grid (Section 2: the cell-centred grid of the
   discrete problem; Section 3.2: its hierarchy of coarser grids); allocates
   the multigrid hierarchy on the device.  stream: a cudaStream_t (NULL =
   default stream).  On success *out receives the context.  Errors: EINVAL
   (bad grid/opts), ENOMEM, ECUDA. */
richards_status richards_create(const richards_grid *grid, const richards_opts *opts,
                                void *stream, richards_ctx **out);

/* Soil law and parameters (Table 1).  EINVAL: Ks <= 0, theta_s <= theta_r,
   theta_r < 0, VG n <= 1, Haverkamp A/alpha/beta/gamma <= 0, Gardner alpha
   <= 0, or a non-finite value in a field. */
richards_status richards_set_soil(richards_ctx *ctx, const richards_soil *soil);

/* Layered soil (Section 4.1's composite law; Section 4.2's two layers): up
   to 8 materials, each a Table 1 law (model, Ks, theta_s, theta_r and p1..p4
   as in richards_soil), and a material index per cell of the finest level
   (host array of ncell bytes, copied; layout as psi).  Every cell then takes
   its material's law and parameters everywhere (theta, theta', K, the point
   solve's bracket, K(psi_b) on a Dirichlet face); conductivities stay
   cell-centred and faces take the mean of the two cell values.  A coarse
   cell takes the material with the largest total restriction weight among
   its fine cells (ties: the lower index) and that material's parameters.
   Replaces the soil set by richards_set_soil (and is replaced by the next
   such call).  Ownership: nothing is retained.  EINVAL: nmat outside 1..8, a
   material failing richards_set_soil's checks, or an index >= nmat. */
typedef struct {
  int model;
  double Ks, theta_s, theta_r, p1, p2, p3, p4;
} richards_material;
richards_status richards_set_materials(richards_ctx *ctx, const richards_material *mats, int nmat,
                                       const unsigned char *index);

/* Boundary conditions (see richards_bc) of the operator of Section 2
   (eq. discrete-strong, written as fluxes: a Dirichlet face contributes a
   half-cell conductance to the diagonal and its head to g; an inflow q/h
   and free drainage -Kc/h go into g).  EINVAL: unknown kind, free drainage
   off the bottom face, non-finite value. */
richards_status richards_set_bc(richards_ctx *ctx, const richards_bc *bc);

/* Sink S(psi) (reading of assumption (A2), Section 2: S non-decreasing on
   its rising branch; Feddes shape times a root-zone profile).  EINVAL: not
   h4 < h3 <= h2 < h1. */
richards_status richards_set_sink(richards_ctx *ctx, const richards_sink *sink);

/* State psi^n (host array, ncell doubles) and, for BDF2, psi^{n-1}
   (nullable: the next BDF2 step then falls back to BDF1): the history of
   eq. fully-bdf1 and of the BDF2 reading.  t: model time.
   EINVAL on a non-finite value (the context is then left as it was).  In
   the mixed modes an array equal bit for bit, cell by cell, to the
   context's current psi^n (psi^{n-1}) keeps the cached theta of that state
   -- the state a caller got from richards_get_state and hands back
   unchanged -- so the next step does not evaluate the law there again; an
   array that differs anywhere replaces the cache (the comparison runs on
   the device, in the same pass as the finiteness check). */
richards_status richards_set_state(richards_ctx *ctx, const double *psi,
                                   const double *psi_prev, double t);

/* One implicit step of size dt: BDF1 (eq. fully-bdf1) for scheme 1, the BDF2
   reading for scheme 2.  Cycles to the tolerance, then shifts the history.
   info (nullable) receives the step statistics.  ENOCONV: psi^{n+1} is the
   last iterate and the history is shifted all the same; ENAN: state rolled
   back to psi^n. */
richards_status richards_step(richards_ctx *ctx, double dt, int scheme,
                              richards_step_info *info);

/* nsteps calls of richards_step (eq. fully-bdf1 or the BDF2 reading, one
   after the other); stops at the first error.  last receives the last
   step's statistics. */
richards_status richards_solve(richards_ctx *ctx, double dt, int nsteps, int scheme,
                               richards_step_info *last);

/* Copy psi^n out.  on_device = 0: psi_out is a host array of ncell doubles;
   1: a device pointer (ordered on the context's stream). */
richards_status richards_get_state(richards_ctx *ctx, double *psi_out, int on_device);

/* Water content and conductivity (Table 1, with each cell's own soil
   parameters) at given pressure heads: theta_out[i] = theta(psi[i]),
   K_out[i] = K(psi[i]) for the ncell cells of the finest level; theta_out or
   K_out may be NULL.  on_device = 0: host arrays; 1: device arrays (ordered
   on the context's stream).  arith 0: FP64, as every step computes them;
   1: float-float (~1e-12 relative), the arithmetic of the mixed mode's
   steering defects.  Returns RICH_EINVAL for a bad arith or before the soil
   is set.  Useful for water-volume (mass balance) accounting. */
richards_status richards_soil_eval(richards_ctx *ctx, const double *psi, double *theta_out,
                                   double *K_out, int arith, int on_device);

/* Model time and number of cells of the finest level. */
double richards_time(const richards_ctx *ctx);
long long richards_ncell(const richards_ctx *ctx);

/* Message describing the last failure on this context (static storage
   owned by the context); "" when none. */
const char *richards_last_error(const richards_ctx *ctx);

/* Why a step of this context launches its FP32 inner cycles one by one
   instead of as CUDA graphs (static storage owned by the context; "" when
   every graph it needed so far was built): the cycle graph (one replay per
   cycle) and the inner-loop graph (the whole inner solve: a conditional
   while node around the cycle and its stop test, so that no cycle waits
   for the host).  Graphs are used on a stream of the context's own
   (not the NULL stream) with opts.graphs set and kernel timing off. */
const char *richards_graph_status(const richards_ctx *ctx);

/* Release the context and all its device memory.  NULL is accepted. */
void richards_destroy(richards_ctx *ctx);

/* ---------------------------------------------------------------------
 * Concurrent requests.  richards_batch_submit starts, for each context, a
 * host worker thread that runs nsteps steps (richards_step: eq. fully-bdf1
 * or the BDF2 reading, Section 3.2's cycles) on the context's stream; the
 * contexts' work overlaps on the device when they have distinct streams.
 * While a context runs, every other call on it returns RICH_EBUSY.
 * --------------------------------------------------------------------- */

/* EINVAL on a NULL or repeated context or bad arguments; EBUSY if one is
   already running (nothing is started then). */
richards_status richards_batch_submit(richards_ctx *const *ctxs, int n, double dt, int nsteps, int scheme);

/* done[k] = 1 when context k has finished (0 while running); for finished
   contexts status[k] and info[k] (both nullable) receive the outcome of the
   run and its statistics: cycles, outer_iters and cell_updates summed over
   the steps, resid0 of the first step, resid and scheme_used of the last. */
richards_status richards_batch_poll(richards_ctx *const *ctxs, int n, int *done, richards_status *status,
                                    richards_step_info *info);

/* The FP64 elementary functions the soil laws use (Table 1's powers and
   exponentials: fn 0 exp, 1 expm1, 2 log, 3 log1p; table-driven, a few ulps
   from the correctly rounded value) or, for comparison, CUDA's own (fn 4..7
   in the same order): y[i] = f(x[i]) for device arrays of n doubles, on the
   given stream (synchronised).  The paper has no counterpart: a check of the
   library's arithmetic.  EINVAL for a bad fn or null arrays. */
richards_status richards_math_eval(int fn, const double *x, double *y, long long n, void *stream);

/* ---------------------------------------------------------------------
 * Launch shapes of the FP32 grid kernels (mixed modes).  The paper has no
 * counterpart: these choose how the kernels of a level are laid out on the
 * GPU, never what they compute (one cell's arithmetic does not depend on the
 * launch shape, so every choice gives the same bits).
 * --------------------------------------------------------------------- */

/* Time, on the context's current prepared state, every candidate shape of
   each grid level with at least 2^15 cells -- cells per thread along z of
   the half-sweeps (1, 2, 4, 8; the finest level keeps 2 where its last
   half-sweep also writes the defects), their block x-size (32..256; 128 at
   most with more than one plane) and the defect kernel's block x-size --
   over reps red+black half-sweeps (defects) each, and keep the fastest; the
   state is restored.  planes_out / bx_out / rbx_out (nullable, nlevels
   entries) receive the choices (0: default).  Needs a mixed-mode context
   (precision 1 or 2) with red-black sweeps after richards_prepare or a
   step.  Errors: EINVAL, EBUSY, ENOMEM (the saved state), ECUDA. */
richards_status richards_autotune(richards_ctx *ctx, int reps, int *planes_out, int *bx_out, int *rbx_out);

/* Set a level's shapes by hand (0 restores a default).  EINVAL outside the
   candidate sets above. */
richards_status richards_set_launch(richards_ctx *ctx, int level, int planes, int block_x, int resid_block_x);

/* FP32 inner cycles: the levels below the finest with at most max_cells
   cells, down to the coarsest, run as one cooperative launch per visit --
   every block of the grid walks the cycle, with a grid barrier between
   stages instead of a launch per stage, and block 0 alone takes the levels
   of the single-block tail.  Same values as the stage launches.  Off (0) by
   default: on the 256^3 drainage the grid barriers cost more than the
   graph-replayed launches they replace.  EINVAL for a negative size. */
richards_status richards_set_coop(richards_ctx *ctx, long long max_cells);

/* ---------------------------------------------------------------------
 * Batched steps of resident contexts (continuous batching of served
 * requests).  A batcher advances many contexts in ticks: at every tick each
 * context does the next part of its own current step -- its preparation and
 * first outer defect, an outer defect and the decision after it, one FP32
 * inner V-cycle, or the step's water balance and history shift -- whatever
 * the other contexts are doing.  The inner V-cycles of all contexts that are
 * in an inner solve run together: every stage of a cycle (half-sweep,
 * defect, restriction, FAS right side, interpolation, coarse tail) is one
 * launch over a device table of (context, level) descriptors on the
 * batcher's stream (Section 3.2's cycle for each context); the work of one
 * context alone runs on the context's own stream and overlaps them.  A
 * context whose finest level has 2^20 cells or more fills the GPU alone: its
 * cycles run as in richards_step (its own cycle graph, on its own stream).  A
 * context's arithmetic, decisions and results are those of richards_step
 * (no reduction mixes contexts).  A context can be mid-step when a call
 * returns; the next call continues it (a call that prepares a step of the
 * context or changes its problem drops that progress: the step restarts
 * from psi^n).  The caller may change the list between calls (admit new
 * requests, retire finished ones).
 * --------------------------------------------------------------------- */
typedef struct richards_batcher richards_batcher;   /* opaque; owns its descriptor tables */

/* stream: the cudaStream_t the batched cycles run on (NULL = default
   stream); max_contexts: the most contexts one call takes (1..4096).
   Errors: EINVAL, ENOMEM. */
richards_status richards_batcher_create(void *stream, int max_contexts, richards_batcher **out);
void richards_batcher_destroy(richards_batcher *b);
const char *richards_batcher_last_error(const richards_batcher *b);

/* One step of each of the n contexts (dt[k], scheme[k]: as richards_step,
   an implicit step of eq. fully-bdf1 or the BDF2 reading solved by Section
   3.2's cycles); returns when all are done.  Every context must be in a mixed mode
   (precision 1 or 2) with red-black sweeps and no FMG start, and all must
   share nu1, nu2, cycle_gamma, gamma_levels, coarse_max_sweeps, coarse_rtol
   and inner_cycles.  Work is ordered after what the contexts' streams hold.
   status[k] / info[k] (nullable) receive each context's outcome as
   richards_step would return it.  Returns EINVAL / EBUSY before doing
   anything when an argument or a context does not qualify, ECUDA on a CUDA
   error (no context is then left mid-step), else RICH_OK. */
richards_status richards_batcher_step(richards_batcher *b, richards_ctx *const *ctxs, int n, const double *dt,
                                      const int *scheme, richards_status *status, richards_step_info *info);

/* Continuous batching: steps_left[k] (host, in/out) more steps of context
   k, each context on its own schedule; returns after max_ticks ticks (> 0;
   0 = no limit) or as soon as a context that wanted steps has done all of
   them (a failed step ends a context's run: its steps_left becomes 0), or
   when no context wants more.  Per context (host arrays, nullable):
   steps_done[k] = steps completed in this call; status[k] = the last one's
   status (RICH_OK if none); info[k] = their statistics: cycles,
   outer_iters and cell_updates summed over them, resid0 from the first,
   the rest from the last.  Same requirements and errors as
   richards_batcher_step; EINVAL for a negative steps_left. */
richards_status richards_batcher_advance(richards_batcher *b, richards_ctx *const *ctxs, int n, const double *dt,
                                         const int *scheme, int *steps_left, int max_ticks, int *steps_done,
                                         richards_status *status, richards_step_info *info);

/* Device memory a context for this grid and these options allocates
   (upper estimate, bytes; no device is touched): soil_fields != 0 when the
   soil has per-cell fields, sink != 0 with a sink.  -1 on invalid input. */
long long richards_device_bytes(const richards_grid *grid, const richards_opts *opts, int soil_fields, int sink);

/* ---------------------------------------------------------------------
 * Inspection and kernel-level entry points.  They run single stages of the
 * step on the context's current data so that each kernel can be checked
 * against the CPU oracle.  Levels count from 0 (finest).
 * --------------------------------------------------------------------- */

/* Per-step set-up without solving: lagged state psi*, Kc = K(psi*), the
   boundary conductances and the right side g of eq. (Nh-def) on the finest
   level, restricted Kc and conductances on coarser levels; the iterate of
   level 0 is set to psi^n.  Returns the scheme used through *scheme_used. */
richards_status richards_prepare(richards_ctx *ctx, double dt, int scheme, int *scheme_used);

int richards_nlevels(const richards_ctx *ctx);
richards_status richards_level_dims(const richards_ctx *ctx, int level, int n_out[3]);

/* Arrays of a level (FP64 copies, host buffers):
     0 iterate psi, 1 right side g, 2 Kc, 3 p1, 4 p2, 5 sink coefficient,
     6 FAS restricted iterate psi_bar, 7 defect d, 8 material index (layered
     soils only, as doubles), 10+f boundary conductance of face f (face
     cells).  set accepts 0 (iterate) and 1 (right side). */
richards_status richards_get_level(richards_ctx *ctx, int level, int which, double *out,
                                   long long n);
richards_status richards_set_level(richards_ctx *ctx, int level, int which, const double *in,
                                   long long n);

/* One red (color 0) or black (color 1) half-sweep of eq. (point-update) on
   a level's iterate with its right side (FP64); color -1: both.  With
   ordering 0 only color -1 is accepted: one lexicographic sweep. */
richards_status richards_sweep(richards_ctx *ctx, int level, int color);

/* d = g - N(psi) on a level (FP64; N of eq. Nh-def, the defect of FAS
   step 2, Section 3.2) into the level's defect; *norm gets ||d||_inf
   (nullable). */
richards_status richards_residual(richards_ctx *ctx, int level, double *norm);

/* FAS steps 2-4 from `level` to level+1: defect, restriction of iterate and
   defect, coarse right side g_H = N_H(psi_bar_H) + d_H, coarse iterate =
   psi_bar_H (FP64). */
richards_status richards_restrict_tau(richards_ctx *ctx, int level);

/* FAS step 6 (Section 3.2): psi_level += P (psi_{level+1} -
   psi_bar_{level+1}) (FP64). */
richards_status richards_prolong(richards_ctx *ctx, int level);

/* One FP64 cycle from the finest level (Section 3.2's recursive FAS cycle;
   the same launches as a step). */
richards_status richards_vcycle(richards_ctx *ctx);

/* ---------------------------------------------------------------------
 * Kernel timing.  While enabled, kernel launches of the context are counted
 * and, depending on the mode, bracketed by CUDA events on the context's
 * stream; richards_profile_read synchronises the stream and returns, per
 * kernel name and level, the number of launches, their summed device time
 * (0 for launches that were only counted) and the cells they covered (a
 * half-sweep covers the cells of one colour).
 * --------------------------------------------------------------------- */
typedef struct {
  char name[32];
  int level;
  long long launches;
  double ms;
  long long cells;
} richards_kernel_stat;

/* enable = 0: stop; otherwise clear the records and start recording:
   1 time every launch; 2 time the finest level's launches and count the
   others; 3 count only (no events, so no timing overhead). */
richards_status richards_profile(richards_ctx *ctx, int enable);

/* Writes up to max records into out; returns the number of records (or -1
   on error). */
int richards_profile_read(richards_ctx *ctx, richards_kernel_stat *out, int max);

/* ---------------------------------------------------------------------
 * Allocation-free step for small grids.  The paper has no counterpart: this
 * is an interface for callers that may not allocate device memory while
 * they run -- programs whose memory pool already holds all of the device
 * memory, real-time loops that forbid allocator calls (an allocation can
 * block and synchronise the device), plug-ins that may only touch memory
 * handed to them.
 *
 * One implicit step (eq. fully-bdf1 or the BDF2 reading, solved by the FAS
 * cycles of Section 3.2 with the point update of eq. point-update: the same
 * arithmetic as richards_step in FP64 mode) of a grid with at most
 * RICHARDS_NOALLOC_MAX_CELLS cells, run in a single thread block.  psi_n, psi_prev (nullable: BDF1 is used) and psi_out are device
 * arrays of ncell doubles; psi_out may alias psi_n or psi_prev (both are
 * read before anything is written).  In this call the optional soil fields
 * (Ks_field, p1_field, p2_field) and boundary fields (value_field,
 * mask_field) are DEVICE pointers.  The soil, boundary and sink parameters
 * are checked as by richards_set_soil / set_bc / set_sink (fields
 * excepted).  The step is FP64 and starts from psi_n with V/W-cycles:
 * opts->precision, ordering (red-black is used), fmg_cycles, predictor,
 * graphs, sweep_planes, tail_cells and the inner_* and max_outer options
 * are ignored.  info (nullable, host) receives the statistics.  stream: a
 * cudaStream_t (NULL = default stream); the call synchronises it.
 *
 * Scratch: one fixed 2 MiB array in the library's device memory (every
 * device that loads the library keeps it until the process exits); nothing
 * is allocated.  The first call on each device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current.  All calls share
 * the array: calls that overlap on the GPU (two streams, two host threads)
 * race and must be serialised by the caller.  The array keeps the last call's
 * contents; a call writes every value before reading it, so nothing has to
 * start at zero.
 *
 * Errors: EINVAL for a grid above RICHARDS_NOALLOC_MAX_CELLS cells (its
 * hierarchy would not fit the fixed scratch) or any invalid argument;
 * ENOCONV / ENAN as for richards_step; ECUDA on a CUDA error. */
#define RICHARDS_NOALLOC_MAX_CELLS 4096
richards_status richards_step_small_noalloc(const richards_grid *grid, const richards_soil *soil,
                                            const richards_bc *bc, const richards_sink *sink,
                                            const richards_opts *opts, double dt, int scheme,
                                            const double *psi_n, const double *psi_prev, double *psi_out,
                                            richards_step_info *info, void *stream);

/* ---------------------------------------------------------------------
 * Batched soil columns: many independent 1D columns of uneven length solved
 * in persistent launches, one per length class (a device work queue per
 * class, longest column first; each thread block runs all time steps of one
 * column with the column's whole multigrid hierarchy in shared memory).  Mixed precision as for
 * richards_step: FP32 FAS cycles on the correction equation inside an outer
 * defect correction whose lagged K, history, defect and stop test run in
 * float-float arithmetic (laws ~1e-12 relative) with opts->precision 1, or
 * in FP64 with opts->precision 2 (float-float defects steer, the FP64 defect
 * decides the stop test); precision 0 is taken as 1.
 * --------------------------------------------------------------------- */
#define RICHARDS_COLUMN_MAX_CELLS 2048
typedef struct richards_columns richards_columns;   /* opaque; owns its device memory */

/* One column: n cells over length L (axis 0 is vertical, face 0 the bottom,
   face 1 the top); scalar soil (fields are ignored; every column of a batch
   uses the same soil law); boundary kinds/values as in richards_bc. */
typedef struct {
  int n;
  double L;
  richards_soil soil;
  int bc_kind[2];
  double bc_value[2];
} richards_column;

/* Create a batch; the sink (reading of (A2)) and the options are shared.
   EINVAL: a column above RICHARDS_COLUMN_MAX_CELLS cells, mixed soil laws,
   invalid parameters; ENOMEM; ECUDA. */
richards_status richards_columns_create(int ncol, const richards_column *cols, const richards_sink *sink,
                                        const richards_opts *opts, void *stream, richards_columns **out);
void richards_columns_destroy(richards_columns *batch);
long long richards_columns_ncell(const richards_columns *batch);

/* States of all columns, packed in column order (host arrays of ncell
   doubles); psi_prev nullable (the next BDF2 step falls back to BDF1). */
richards_status richards_columns_set_state(richards_columns *batch, const double *psi, const double *psi_prev);

/* nsteps implicit steps of every column (scheme 1 = BDF1 of eq.
   fully-bdf1, 2 = the BDF2 reading; Section 4.1's column problem, solved by
   the FAS cycles of Section 3.2): one persistent launch per length class
   (columns of more than 512 cells, 257-512, at most 256; the two shorter
   classes on streams of the batch's own, joined to its stream by events);
   returns once all are done.
   Per-column outcomes are read with richards_columns_stats. */
richards_status richards_columns_run(richards_columns *batch, double dt, int nsteps, int scheme);

richards_status richards_columns_get_state(richards_columns *batch, double *psi, int on_device);

/* Per column (host arrays of ncol entries, each nullable): status of the
   last run (RICH_OK / ENOCONV / ENAN), FP32 inner cycles, outer (float-float defect)
   iterations, last tau_eff ||g - N(psi)||_inf, NGS point updates. */
richards_status richards_columns_stats(richards_columns *batch, int *status, int *cycles, int *outer,
                                       double *resid, long long *updates);

/* Threads per block of the longest class (64, 128, 256 or 512); the next
   classes take a half and a quarter of it (at least 32).  Results do not
   depend on it. */
richards_status richards_columns_set_threads(richards_columns *batch, int threads);

/* For each block size (128, 256, 512): one untimed step, then two timed
   steps of every column from the same state; keeps the fastest and restores
   the state.  *threads_out (nullable) gets it. */
richards_status richards_columns_autotune(richards_columns *batch, double dt, int scheme, int *threads_out);

#ifdef __cplusplus
}
#endif
#endif
