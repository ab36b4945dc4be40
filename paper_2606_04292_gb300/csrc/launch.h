// Host-callable launchers of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "richards.h"

#include "ddmath.cuh"
#include "device.cuh"

#define TAIL_THREADS 512

namespace rich {

struct BcDev {
  int kind[6];
  double value[6];
  const double* vfield[6];
  const unsigned char* mask[6];
};

struct Geom {
  int dim, n0, n1, n2;
  double h[3];
  double Lv;            // length of the vertical axis
};

// FP64, psi as unknown
void sweep64(const Level<double>& L, const Phys<double>& P, int model, int color, cudaStream_t s);
void residual64(const Level<double>& L, const Phys<double>& P, int model, unsigned long long* norm,
                cudaStream_t s);
void tau64(const Level<double>& C, const Phys<double>& P, int model, cudaStream_t s);
void restrict64(const Level<double>& F, const Level<double>& C, const Xfer<double>& X, const double* fa,
                const double* fb, double* ca, double* cb, cudaStream_t s);
void prolong64(const Level<double>& F, const Level<double>& C, const Xfer<double>& X, cudaStream_t s);
// ordering: 1 red-black, 0 lexicographic (hyperplane by hyperplane)
void tail64(const Level<double>* dLs, const Xfer<double>* dXs, int l0, int nl, const Phys<double>& P,
            int model, int nu1, int nu2, int cmax, double crtol, int gamma, int gamma_levels,
            unsigned long long* stats, int ordering, cudaStream_t s);
// one lexicographic NGS sweep (a launch per hyperplane i0 + i1 + i2 = const)
void sweep_lex64(const Level<double>& L, const Phys<double>& P, int model, cudaStream_t s);

// FP32, correction delta as unknown
// (bx > 0: the block x-size and, for sweeps, the pipelined kernel below 2^20
// cells too, as the autotuner chose them; 0: the defaults)
void sweep32(const Level<float>& L, const Phys<float>& P, int model, int color, int planes, cudaStream_t s,
             int bx = 0);
void residual32(const Level<float>& L, const Phys<float>& P, int model, unsigned long long* norm,
                cudaStream_t s, int bx = 0);
void tau32(const Level<float>& C, const Phys<float>& P, int model, cudaStream_t s);
// (cs_mask: bit 0 / 1 when fa / fb is a colour-split parameter array of F)
void restrict32(const Level<float>& F, const Level<float>& C, const Xfer<float>& X, const float* fa,
                const float* fb, float* ca, float* cb, cudaStream_t s, int cs_mask = 0);
void prolong32(const Level<float>& F, const Level<float>& C, const Xfer<float>& X, cudaStream_t s);
void tail32(const Level<float>* dLs, const Xfer<float>* dXs, int l0, int nl, const Phys<float>& P,
            int model, int nu1, int nu2, int cmax, float crtol, int gamma, int gamma_levels,
            unsigned long long* stats, int ordering, cudaStream_t s);
void sweep_lex32(const Level<float>& L, const Phys<float>& P, int model, cudaStream_t s);
// the cycle from level l0 down as one cooperative launch of `blocks` blocks
// (levels from tail_start on take the single-block tail's transfers); slots:
// three device words for its reductions; stats: its update count
constexpr int COOP_THREADS = 256;
int coop_max_blocks32(int model);
cudaError_t coop32(const Level<float>* dLs, const Xfer<float>* dXs, int l0, int nl, int tail_start,
                   const Phys<float>& P, int model, int nu1, int nu2, int cmax, float crtol, int gamma,
                   int gamma_levels, unsigned long long* stats, unsigned long long* slots, int blocks,
                   cudaStream_t s);
// the last (colour 1) half-sweep of a smoothing that also writes its cells' defects and their
// max into *norm (pipelined two-plane levels only: resid_fusable32), and the defects of one colour
bool resid_fusable32(const Level<float>& L, int planes);
void sweep_resid32(const Level<float>& L, const Phys<float>& P, int model, unsigned long long* norm,
                   cudaStream_t s);
void residual_color32(const Level<float>& L, const Phys<float>& P, int model, int color, unsigned long long* norm,
                      cudaStream_t s);

// per-step preparation (FP64).  mat: the fine level's material index (read
// only when model == COMPOSITE; nullable otherwise)
void prep_lagged(const Geom& G, const double* psin, const double* psinm1, const double* Ks, double Ks_s,
                 const double* p1, const double* p2, const uint8_t* mat, const Phys<double>& P, int model, int scheme,
                 double dt, double* Kc, float* Kcf, double* g, double* u, const double* thn_in,
                 const double* thm_in, double* thn_out, double* thm_out, bool predict, cudaStream_t s,
                 const double* vgm = nullptr);
void prep_rhs(const Geom& G, const BcDev& bc, const double* Ks, double Ks_s, const double* p1, const double* p2,
              const uint8_t* mat, const Phys<double>& P, int model, const double* Kc, double* g, double* const kb[6],
              cudaStream_t s);
// mixed mode: the same terms in float-float
void prep_rhs_dd(const Geom& G, const BcDev& bc, const double* Ks, double Ks_s, const double* p1, const double* p2,
                 const uint8_t* mat, const Phys<double>& P, const DDPhys& Q, int model, const double* Kc, double* g,
                 double* const kb[6], cudaStream_t s);
void restrict_face64(const Geom& F, const Geom& C, const Xfer<double>& X, int axis, const double* fine,
                     double* coarse, cudaStream_t s);
void sink_coef(const Geom& G, double Tp, double depth, double decay, double* smax, cudaStream_t s);
void to_float(const double* src, float* dst, long long n, cudaStream_t s);

// mixed mode: r = g - N(u) in float-float -> r32, psi0 = (float)u, delta = 0;
// ||r||_inf as float bits.  theta(u) from th_in if given, else evaluated and
// written to th_out (nullable).
// (cs: r32 and psi0f in the colour-split layout of the FP32 level 0)
void outer_residual_dd(const Level<double>& L, const Phys<double>& P, const DDPhys& Q, int model, float* r32,
                       float* psi0f, float* delta, unsigned long long* norm, const double* th_in, double* th_out,
                       int cs, cudaStream_t s);
// FP64-outer mixed mode: r = g - N(u) in FP64 -> r32, psi0 = (float)u,
// delta = 0; ||r||_inf as FP64 bits; theta caches as outer_residual_dd.
void outer_residual64(const Level<double>& L, const Phys<double>& P, int model, float* r32, float* psi0f,
                      float* delta, unsigned long long* norm, const double* th_in, double* th_out, int cs,
                      cudaStream_t s, const double* vgm = nullptr);
// (vgm, nullable: m = 1 - 1/n of the finest level's van Genuchten n field,
// read instead of divided per cell; vg_m_field makes it)
void vg_m_field(const double* n, double* m, long long count, cudaStream_t s);
// FP32 copy of a level-0 parameter array in the FP32 level's layout (cs: colour-split)
void to_float_level(const double* src, float* dst, int n0, int n1, int n2, int cs, cudaStream_t s);
// natural-layout copy of a colour-split array (the defect at delta = 0 is g)
void cs_to_natural(const float* src, float* dst, int n0, int n1, int n2, cudaStream_t s);
// mixed mode: the lagged state in float-float (Kc to FP64 and FP32)
// (predict: u = psi* instead of psi^n)
void prep_lagged_dd(const Geom& G, const double* psin, const double* psinm1, const double* Ks, double Ks_s,
                    const double* p1, const double* p2, const uint8_t* mat, const Phys<double>& P, const DDPhys& Q,
                    int model, int scheme, double dt, double* Kc, float* Kcf, double* g, double* u,
                    const double* thn_in, const double* thm_in, double* thn_out, double* thm_out, bool predict,
                    cudaStream_t s);
// water balance of a step: per-block partial sums into part (returns the
// block count) and min_i(a theta' + S' + xi) as float bits into *dmin_bits;
// fp64: FP64 laws and sums, else float-float
int mass_balance(const Level<double>& L, const Geom& G, const BcDev& bc, const Phys<double>& P, const Phys<float>& Pf,
                 int model, const double* psin, const double* psinm1, int scheme, double dt, const double* th_new,
                 const double* th_n, const double* th_nm1, double* part, unsigned* dmin_bits, bool fp64,
                 cudaStream_t s);
void restrict_face32(const Geom& F, const Geom& C, const Xfer<float>& X, int axis, const float* fine, float* coarse,
                     cudaStream_t s);
void apply_delta(double* u, const float* delta, long long n, cudaStream_t s);
// y = f(x) elementwise for the laws' FP64 elementary functions (fn 0..3:
// exp, expm1, log, log1p) or CUDA's (fn 4..7), device arrays
void math_eval(int fn, const double* x, double* y, long long n, cudaStream_t s);
// *flags |= 1 if any of x[0..n) is NaN or infinite, and, with ref non-null,
// *flags |= changed_bit if any x[i] differs from ref[i] bit for bit
void screen_state(const double* x, const double* ref, long long n, unsigned changed_bit, unsigned* flags,
                  cudaStream_t s);
// theta(psi) and K(psi) per cell (FP64 or float-float); outputs nullable
void soil_eval(long long n, const double* psi, const double* Ks, double Ks_s, const double* p1, const double* p2,
               const uint8_t* mat, const Phys<double>& P, const DDPhys& Q, int model, bool dd, double* theta,
               double* K, cudaStream_t s);

}  // namespace rich

// ---------------------------------------------------------------------------
// Batched FP32 inner cycles (batch.cu): one launch runs one stage of the
// cycle on one level of every context in a list.  The device table holds a
// descriptor per (context, level); a list names the descriptors of a launch
// and the first block of each (blocks of BATCH_THREADS threads, laid out
// per descriptor as the single-context launch lays out its grid).
// ---------------------------------------------------------------------------
namespace rich {

constexpr int BATCH_THREADS = 128;
constexpr int BATCH_MAX = 64;        // descriptors per launch

struct BJob32 {
  Level<float> F, C;                 // the level and the next coarser one (C unused on the coarsest)
  Xfer<float> X;                     // transfers between them
  Phys<float> P;
  const Level<float>* dLs;           // the context's device level views (coarse tail)
  const Xfer<float>* dXs;
  int level, nlev;
  int model;                         // the context's law (HAVERKAMP, GARDNER, VANGENUCHTEN, COMPOSITE)
  unsigned long long* norm;          // the context's inner-norm slot (float bits)
  unsigned long long* stats;         // the context's coarse-tail update counter
};

struct BList {
  int n;
  int job[BATCH_MAX];                // table index of each descriptor
  int block0[BATCH_MAX + 1];         // first block of each; block0[n] = total
};

enum { BOP_SWEEP = 0, BOP_RESID = 1, BOP_RESTRICT = 2, BOP_TAU = 3, BOP_PROLONG = 4 };

// blocks one descriptor takes for a stage
int batch_blocks(int op, const BJob32& j);
// one stage over the listed descriptors, of any laws (each block branches on
// its descriptor's), all with one fixed Newton count nk: 1, 2, or 0 for
// P.newton_k; color for BOP_SWEEP; with_norm: the defect's max into each
// descriptor's norm slot (BOP_RESID)
void batch32(int op, int nk, const BJob32* table, const BList& list, int color, bool with_norm, cudaStream_t s);
// the coarse tail from each listed descriptor's level: one block each
void batch_tail32(const BJob32* table, const BList& list, int nu1, int nu2, int cmax, float crtol, int gamma,
                  int gamma_levels, cudaStream_t s);

}  // namespace rich

// ---------------------------------------------------------------------------
// One FP64 step of a small grid in a single thread block (noalloc.cu): the
// allocation-free entry point and contexts whose grid fits one block use it.
// ---------------------------------------------------------------------------
namespace rich {

// a context's hierarchy: level views (every array, material maps included),
// transfer tables, material table (layered soils)
struct SmallCtx {
  int nlev;
  const Level<double>* L;
  const Xfer<double>* X;
  const MatLaw<double>* mats;
};

// one step on the context's own levels (soil and bc fields are device
// arrays); only the 32 doubles of statistics at stats_dev are extra; ordering
// 1 red-black, 0 lexicographic; stats_out (host, 5 doubles): cycles, resid0,
// resid, status, updates; synchronises s
richards_status small_step(const richards_grid* grid, const richards_soil* soil, const richards_bc* bc,
                           const richards_sink* sink, const richards_opts* opts, double dt, int scheme,
                           const double* psi_n, const double* psi_prev, double* psi_out, double* stats_dev,
                           const SmallCtx* cx, int ordering, double* stats_out, cudaStream_t s);

}  // namespace rich
