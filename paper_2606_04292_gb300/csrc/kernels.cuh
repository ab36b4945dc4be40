// Grid kernels of one V-cycle level and the single-block coarse tail.
// Included by the FP64 and FP32 translation units, which instantiate them.
#pragma once

#include <algorithm>

#include <cooperative_groups.h>

#include "device.cuh"
#include "launch.h"

namespace rich {

template <typename T>
__device__ __forceinline__ T from_bits(unsigned long long b);
template <>
__device__ __forceinline__ double from_bits<double>(unsigned long long b) {
  return __longlong_as_double((long long)b);
}
template <>
__device__ __forceinline__ float from_bits<float>(unsigned long long b) {
  return __uint_as_float((unsigned)b);
}

// ---------------------------------------------------------------------------
// One colour of a red-black NGS sweep (eq. point-update for every cell of the
// colour; cells of one colour do not couple, so the update is parallel).
// ---------------------------------------------------------------------------
// Launch grid: x = pairs of cells along a row, y = row, z = plane.
// (The bodies of the grid kernels take the block's coordinates explicitly:
// the batched kernels run the same bodies for the blocks of many grids.)
template <typename T, int FORM, int MODEL, int NK = 0>
__device__ __forceinline__ void sweep_body(const Level<T>& L, const Phys<T>& P, int color, int bx, int by, int bz) {
  const int p = bx * blockDim.x + threadIdx.x;
  const int i1 = by, i2 = bz;
  const int i0 = 2 * p + ((color + i1 + i2) & 1);
  if (i0 >= L.n0) return;
  const long long i = (unsigned)(i0 + L.n0 * (i1 + L.n1 * i2));
  point_update<T, FORM, MODEL, NK>(L, P, i, i0, i1, i2);
}

template <typename T, int FORM, int MODEL, int NK = 0>
__global__ void __launch_bounds__(256) k_sweep(Level<T> L, Phys<T> P, int color) {
  sweep_body<T, FORM, MODEL, NK>(L, P, color, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The same half-sweep with ZC planes per thread, software-pipelined: the
// operands of the next plane's cell are loaded before the current cell is
// solved.  Launch grid: x = pairs of cells along a row, y = row, z = chunk
// of ZC planes.
// RESID: the half-sweep also writes the defect d = g - N(u) of each cell it
// updates, at the new value (its neighbours, of the other colour, do not
// change during the half-sweep), and returns the largest |d| (bits)
template <typename T, int FORM, int MODEL, int ZC, int NK, bool YZI, bool RESID>
__device__ __forceinline__ unsigned long long sweep_pipe_body(const Level<T>& L, const Phys<T>& P, int color, int p,
                                                              int i1, int z0) {
  unsigned long long mx = 0;
  CellOps<T> c[2];
  {
    const int i0 = 2 * p + ((color + i1 + z0) & 1);
    c[0].valid = z0 < L.n2 && i0 < L.n0;
    if (c[0].valid) gather<T, FORM, MODEL, YZI>(L, P, i0, i1, z0, c[0]);
  }
#pragma unroll
  for (int k = 0; k < ZC; ++k) {
    if (k + 1 < ZC) {
      const int i2 = z0 + k + 1;
      const int i0 = 2 * p + ((color + i1 + i2) & 1);
      CellOps<T>& nx = c[(k + 1) & 1];
      nx.valid = i2 < L.n2 && i0 < L.n0;
      if (nx.valid) gather<T, FORM, MODEL, YZI>(L, P, i0, i1, i2, nx);
    }
    const CellOps<T>& cur = c[k & 1];
    if (cur.valid) {
      T dg, of;
      cell_sums<T, YZI>(L, cur, dg, of);
      const T x = solve_cell_sums<T, FORM, MODEL, NK, YZI>(L, P, cur, dg, of);
      L.u[cur.i] = x;
      if (RESID) {
        const T di = cell_defect<T, FORM, MODEL>(P, cur, dg, of, x);
        L.d[cur.i] = di;
        const unsigned long long b = nbits(di);
        mx = b > mx ? b : mx;
      }
    }
  }
  return mx;
}

template <typename T, int FORM, int MODEL, int ZC, int NK = 0, bool RESID = false>
__global__ void __launch_bounds__(128) k_sweep_pipe(Level<T> L, Phys<T> P, int color, unsigned long long* norm) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int i1 = blockIdx.y;
  const int z0 = blockIdx.z * ZC;
  // blocks away from the y and z boundaries (all but a thin shell) skip
  // those boundary tests; the branch is uniform over the block
  // (the deeper pipelines, 4 and 8 planes, keep one body: compile time)
  unsigned long long mx;
  if constexpr (ZC == 2) {
    const bool yzi = L.dim == 3 && i1 > 0 && i1 < L.n1 - 1 && z0 > 0 && z0 + ZC < L.n2;
    mx = yzi ? sweep_pipe_body<T, FORM, MODEL, ZC, NK, true, RESID>(L, P, color, p, i1, z0)
             : sweep_pipe_body<T, FORM, MODEL, ZC, NK, false, RESID>(L, P, color, p, i1, z0);
  } else {
    mx = sweep_pipe_body<T, FORM, MODEL, ZC, NK, false, RESID>(L, P, color, p, i1, z0);
  }
  if (RESID) {
    __shared__ unsigned long long sm[33];
    mx = block_max(mx, sm);
    if (threadIdx.x == 0) atomicMax(norm, mx);
  }
}

// The defect of the cells of one colour (the other colour's defects come
// from a RESID half-sweep).  Launch grid: as k_sweep.
template <typename T, int FORM, int MODEL>
__global__ void __launch_bounds__(256) k_residual_color(Level<T> L, Phys<T> P, int color, unsigned long long* norm) {
  __shared__ unsigned long long sm[33];
  unsigned long long mx = 0;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int i1 = blockIdx.y, i2 = blockIdx.z;
  const int i0 = 2 * p + ((color + i1 + i2) & 1);
  if (i0 < L.n0) {
    const long long i = (unsigned)(i0 + L.n0 * (i1 + L.n1 * i2));
    const bool yzi = L.dim == 3 && i1 > 0 && i1 < L.n1 - 1 && i2 > 0 && i2 < L.n2 - 1;
    const T di = L.g[pix(L, i, i0, i1, i2)] - (yzi ? apply_N<T, FORM, MODEL, true>(L, P, L.u, i, i0, i1, i2)
                                                    : apply_N<T, FORM, MODEL, false>(L, P, L.u, i, i0, i1, i2));
    L.d[i] = di;
    mx = nbits(di);
  }
  mx = block_max(mx, sm);
  if (threadIdx.x == 0) atomicMax(norm, mx);
}

// One hyperplane i0 + i1 + i2 = s of a lexicographic NGS sweep (the
// paper's ordering, Section 3.1: cells in the order of the flattened index).
// Cells of one hyperplane do not couple; each reads the updated values of its
// lower neighbours (plane s - 1) and the old values of its upper ones (plane
// s + 1), exactly what the sequential sweep reads.  Planes s = 0 .. n0+n1+n2-3
// in turn make one sweep.  Launch grid: x = i1, y = i2 - i2lo.
template <typename T, int FORM, int MODEL, int NK = 0>
__global__ void __launch_bounds__(128) k_sweep_plane(Level<T> L, Phys<T> P, int s, int i2lo) {
  const int i1 = blockIdx.x * blockDim.x + threadIdx.x;
  const int i2 = i2lo + blockIdx.y;
  if (i1 >= L.n1) return;
  const int i0 = s - i1 - i2;
  if (i0 < 0 || i0 >= L.n0) return;
  const long long i = (unsigned)(i0 + L.n0 * (i1 + L.n1 * i2));
  point_update<T, FORM, MODEL, NK>(L, P, i, i0, i1, i2);
}

// d = g - N(u) on a level, with ||d||_inf accumulated into *norm (bit max).
// Launch grid: x = cells along a row, y = row, z = plane.
// (returns |d| of the thread's cell as bits, 0 without one)
template <typename T, int FORM, int MODEL>
__device__ __forceinline__ unsigned long long residual_body(const Level<T>& L, const Phys<T>& P, int bx, int by,
                                                            int bz) {
  const int i0 = bx * blockDim.x + threadIdx.x;
  const int i1 = by, i2 = bz;
  if (i0 >= L.n0) return 0;
  const long long i = (unsigned)(i0 + L.n0 * (i1 + L.n1 * i2));
  // rows away from the y/z boundaries skip those tests (uniform over the block)
  const bool yzi = L.dim == 3 && i1 > 0 && i1 < L.n1 - 1 && i2 > 0 && i2 < L.n2 - 1;
  const T di = L.g[pix(L, i, i0, i1, i2)] - (yzi ? apply_N<T, FORM, MODEL, true>(L, P, L.u, i, i0, i1, i2)
                                                  : apply_N<T, FORM, MODEL, false>(L, P, L.u, i, i0, i1, i2));
  L.d[i] = di;
  return nbits(di);
}

template <typename T, int FORM, int MODEL>
__global__ void __launch_bounds__(256) k_residual(Level<T> L, Phys<T> P, unsigned long long* norm) {
  __shared__ unsigned long long sm[33];
  unsigned long long mx = residual_body<T, FORM, MODEL>(L, P, blockIdx.x, blockIdx.y, blockIdx.z);
  if (norm) {
    mx = block_max(mx, sm);
    if (threadIdx.x == 0) atomicMax(norm, mx);
  }
}

// FAS step 3: psi_bar_H = R psi_h, d_H = R d_h (cb may be null).
// (cs_mask: bit 0 / bit 1 set when fa / fb is a colour-split parameter array)
template <typename T>
__device__ __forceinline__ void restrict_body(const Level<T>& F, const Level<T>& C, const Xfer<T>& X, const T* fa,
                                              const T* fb, T* ca, T* cb, int bx, int by, int bz, int cs_mask = 0) {
  const int J0 = bx * blockDim.x + threadIdx.x;
  const int J1 = by, J2 = bz;
  if (J0 >= C.n0) return;
  const long long J = J0 + (long long)C.n0 * (J1 + C.n1 * J2);
  ca[J] = restrict_at(F, X, fa, J0, J1, J2, (cs_mask & 1) != 0);
  if (cb) cb[J] = restrict_at(F, X, fb, J0, J1, J2, (cs_mask & 2) != 0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict(Level<T> F, Level<T> C, Xfer<T> X, const T* fa, const T* fb,
                                                  T* ca, T* cb, int cs_mask) {
  restrict_body<T>(F, C, X, fa, fb, ca, cb, blockIdx.x, blockIdx.y, blockIdx.z, cs_mask);
}

// FAS step 4 on the coarse level: g_H = N_H(psi_bar_H) + d_H, psi_H = psi_bar_H.
template <typename T, int FORM, int MODEL>
__device__ __forceinline__ void tau_body(const Level<T>& C, const Phys<T>& P, int bx, int by, int bz) {
  const int J0 = bx * blockDim.x + threadIdx.x;
  const int J1 = by, J2 = bz;
  if (J0 >= C.n0) return;
  const long long J = J0 + (long long)C.n0 * (J1 + C.n1 * J2);
  // rows away from the y/z boundaries skip those tests (uniform over the block)
  const bool yzi = C.dim == 3 && J1 > 0 && J1 < C.n1 - 1 && J2 > 0 && J2 < C.n2 - 1;
  C.g[J] = (yzi ? apply_N<T, FORM, MODEL, true>(C, P, C.ubar, J, J0, J1, J2)
                : apply_N<T, FORM, MODEL, false>(C, P, C.ubar, J, J0, J1, J2)) + C.d[J];
  C.u[J] = C.ubar[J];
}

template <typename T, int FORM, int MODEL>
__global__ void __launch_bounds__(256) k_tau(Level<T> C, Phys<T> P) {
  tau_body<T, FORM, MODEL>(C, P, blockIdx.x, blockIdx.y, blockIdx.z);
}

// FAS step 6: u_h += P (u_H - psi_bar_H).
template <typename T>
__device__ __forceinline__ void prolong_body(const Level<T>& F, const Level<T>& C, const Xfer<T>& X, int bx, int by,
                                             int bz) {
  const int i0 = bx * blockDim.x + threadIdx.x;
  const int i1 = by, i2 = bz;
  if (i0 >= F.n0) return;
  const long long i = i0 + (long long)F.n0 * (i1 + F.n1 * i2);
  F.u[i] += prolong_at(C, X, i0, i1, i2);
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong(Level<T> F, Level<T> C, Xfer<T> X) {
  prolong_body<T>(F, C, X, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// Nested levels (n_fine = 2 n_coarse on every axis the grid has): the same
// transfer operators with their weights written out, so a thread reads no
// tables.  Restriction taps per axis at fine 2J-1 .. 2J+2 with weights
// (1,3,3,1)/8, at the ends (0,4,3,1)/8 and (1,3,4,0)/8 (the normalised
// transpose of the constant-extrapolation interpolation); an axis of one
// cell is a single tap of weight 1.  Interpolation of an interior fine cell
// i: 3/4 of coarse floor(i/2) and 1/4 of the coarse neighbour on i's side;
// fine end cells take their weights from the tables (they fold the ghost).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void restrict_taps(int J, int nc, int nf, int* idx, T* w) {
  if (nf == 1) {
#pragma unroll
    for (int t = 0; t < 4; ++t) { idx[t] = 0; w[t] = T(0); }
    w[1] = T(1);
    return;
  }
  w[0] = T(0.125); w[1] = T(0.375); w[2] = T(0.375); w[3] = T(0.125);
  if (J == 0) { w[0] = T(0); w[1] = T(0.5); }
  if (J == nc - 1) { w[2] = T(0.5); w[3] = T(0); }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int f = 2 * J - 1 + t;
    idx[t] = f < 0 ? 0 : (f >= nf ? nf - 1 : f);
  }
}

template <typename T>
__device__ __forceinline__ void restrict_nested_body(const Level<T>& F, const Level<T>& C, const T* fa, const T* fb,
                                                     T* ca, T* cb, int bx, int by, int bz, int cs_mask = 0) {
  const int J0 = bx * blockDim.x + threadIdx.x;
  const int J1 = by, J2 = bz;
  if (J0 >= C.n0) return;
  int x[4], y[4], z[4];
  T wx[4], wy[4], wz[4];
  restrict_taps<T>(J0, C.n0, F.n0, x, wx);
  restrict_taps<T>(J1, C.n1, F.n1, y, wy);
  restrict_taps<T>(J2, C.n2, F.n2, z, wz);
  T sa = T(0), sb = T(0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (wz[c] == T(0)) continue;
    T ya = T(0), yb = T(0);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (wy[b] == T(0)) continue;
      const unsigned row = (unsigned)F.n0 * ((unsigned)y[b] + (unsigned)F.n1 * (unsigned)z[c]);
      unsigned ia[4], ib[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ia[a] = row + x[a];
        ib[a] = row + x[a];
        if (cs_mask) {
          const unsigned q = pix_of(1, F.n0, F.n1, F.n2, row + x[a], x[a], y[b], z[c]);
          if (cs_mask & 1) ia[a] = q;
          if (cs_mask & 2) ib[a] = q;
        }
      }
      T xa = T(0);
#pragma unroll
      for (int a = 0; a < 4; ++a) xa += wx[a] * fa[ia[a]];
      ya += wy[b] * xa;
      if (fb) {
        T xb = T(0);
#pragma unroll
        for (int a = 0; a < 4; ++a) xb += wx[a] * fb[ib[a]];
        yb += wy[b] * xb;
      }
    }
    sa += wz[c] * ya;
    sb += wz[c] * yb;
  }
  const unsigned J = (unsigned)(J0 + C.n0 * (J1 + C.n1 * J2));
  ca[J] = sa;
  if (cb) cb[J] = sb;
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_nested(Level<T> F, Level<T> C, const T* fa, const T* fb, T* ca,
                                                         T* cb, int cs_mask) {
  restrict_nested_body<T>(F, C, fa, fb, ca, cb, blockIdx.x, blockIdx.y, blockIdx.z, cs_mask);
}

template <typename T>
__device__ __forceinline__ void prolong_taps(const Xfer<T>& X, int a, int i, int nf, int* j, T* w) {
  if (i > 0 && i < nf - 1) {
    const int J = i >> 1;
    j[0] = J;
    w[0] = T(0.75);
    j[1] = (i & 1) ? J + 1 : J - 1;
    w[1] = T(0.25);
    return;
  }
  const int c = X.pc[a][i];
  j[0] = X.pj[a][2 * i];
  w[0] = X.pw[a][2 * i];
  j[1] = c > 1 ? X.pj[a][2 * i + 1] : j[0];
  w[1] = c > 1 ? X.pw[a][2 * i + 1] : T(0);
}

// the interpolated coarse correction of fine cell (i0, i1, i2), nested levels
template <typename T>
__device__ __forceinline__ T prolong_nested_at(const Level<T>& F, const Level<T>& C, const Xfer<T>& X, int i0, int i1,
                                               int i2) {
  int jx[2], jy[2], jz[2];
  T wx[2], wy[2], wz[2];
  prolong_taps<T>(X, 0, i0, F.n0, jx, wx);
  prolong_taps<T>(X, 1, i1, F.n1, jy, wy);
  prolong_taps<T>(X, 2, i2, F.n2, jz, wz);
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (wz[c] == T(0)) continue;
    T sy = T(0);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (wy[b] == T(0)) continue;
      const unsigned row = (unsigned)C.n0 * ((unsigned)jy[b] + (unsigned)C.n1 * (unsigned)jz[c]);
      T sx = T(0);
#pragma unroll
      for (int a = 0; a < 2; ++a) sx += wx[a] * (C.u[row + jx[a]] - C.ubar[row + jx[a]]);
      sy += wy[b] * sx;
    }
    s += wz[c] * sy;
  }
  return s;
}

template <typename T>
__device__ __forceinline__ void prolong_nested_body(const Level<T>& F, const Level<T>& C, const Xfer<T>& X, int bx,
                                                    int by, int bz) {
  const int i0 = bx * blockDim.x + threadIdx.x;
  const int i1 = by, i2 = bz;
  if (i0 >= F.n0) return;
  const unsigned i = (unsigned)(i0 + F.n0 * (i1 + F.n1 * i2));
  F.u[i] += prolong_nested_at(F, C, X, i0, i1, i2);
}

// one coarse value of the nested full-weighting restriction of a natural
// layout array (the arithmetic of restrict_nested_body, one array)
template <typename T>
__device__ __forceinline__ T restrict_nested_at(const Level<T>& F, const Level<T>& C, const T* fa, int J0, int J1,
                                                int J2) {
  int x[4], y[4], z[4];
  T wx[4], wy[4], wz[4];
  restrict_taps<T>(J0, C.n0, F.n0, x, wx);
  restrict_taps<T>(J1, C.n1, F.n1, y, wy);
  restrict_taps<T>(J2, C.n2, F.n2, z, wz);
  T sa = T(0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (wz[c] == T(0)) continue;
    T ya = T(0);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (wy[b] == T(0)) continue;
      const unsigned row = (unsigned)F.n0 * ((unsigned)y[b] + (unsigned)F.n1 * (unsigned)z[c]);
      T xa = T(0);
#pragma unroll
      for (int a = 0; a < 4; ++a) xa += wx[a] * fa[row + x[a]];
      ya += wy[b] * xa;
    }
    sa += wz[c] * ya;
  }
  return sa;
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_nested(Level<T> F, Level<T> C, Xfer<T> X) {
  prolong_nested_body<T>(F, C, X, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// The interpolation of big 3-d levels through a shared-memory tile: a block
// first stages, in coalesced rows, the coarse corrections u_H - psi_bar_H its
// fine tile reads, with a one-cell halo (out-of-range halo cells repeat the
// edge and are never weighted), then evaluates the taps of
// k_prolong_nested, in the same order, from shared memory: same results,
// fewer L1 requests (16 global loads per fine cell become 8 shared ones).
// (The same staging for the restriction measured slower than its L1-cached
// kernel: 64 taps per coarse cell reuse the cache well.)
// ---------------------------------------------------------------------------
template <typename T>
struct TransferTile {
  static constexpr int PX = 64, PY = 4, PZ = 4;                         // fine tile of the interpolation
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename T>
__global__ void __launch_bounds__(TransferTile<T>::PX * TransferTile<T>::PY)
k_prolong_tiled(Level<T> F, Level<T> C, Xfer<T> X) {
  constexpr int PX = TransferTile<T>::PX, PY = TransferTile<T>::PY, PZ = TransferTile<T>::PZ;
  constexpr int CX = PX / 2 + 2, CY = PY / 2 + 2, CZ = PZ / 2 + 2, NT = PX * PY;
  __shared__ T se[CZ][CY][CX];
  const int x0 = blockIdx.x * PX, y0 = blockIdx.y * PY, z0 = blockIdx.z * PZ;
  const int cx0 = x0 / 2 - 1, cy0 = y0 / 2 - 1, cz0 = z0 / 2 - 1;
  for (int t = threadIdx.x; t < CX * CY * CZ; t += NT) {
    const int x = t % CX, y = (t / CX) % CY, z = t / (CX * CY);
    const int gx = clampi(cx0 + x, 0, C.n0 - 1), gy = clampi(cy0 + y, 0, C.n1 - 1), gz = clampi(cz0 + z, 0, C.n2 - 1);
    const unsigned gj = (unsigned)gx + (unsigned)C.n0 * ((unsigned)gy + (unsigned)C.n1 * (unsigned)gz);
    se[z][y][x] = C.u[gj] - C.ubar[gj];
  }
  __syncthreads();
  const int i0 = x0 + threadIdx.x % PX, i1 = y0 + threadIdx.x / PX;
  if (i0 >= F.n0 || i1 >= F.n1) return;
  int jx[2], jy[2];
  T wx[2], wy[2];
  prolong_taps<T>(X, 0, i0, F.n0, jx, wx);
  prolong_taps<T>(X, 1, i1, F.n1, jy, wy);
  // the x-y interpolation of each staged coarse plane, once for the PZ fine
  // cells of the column that share it (the sums of prolong_nested_at)
  T py[CZ];
#pragma unroll
  for (int p = 0; p < CZ; ++p) {
    T sy = T(0);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (wy[b] == T(0)) continue;
      const T* row = &se[p][jy[b] - cy0][0];
      T sx = T(0);
#pragma unroll
      for (int a = 0; a < 2; ++a) sx += wx[a] * row[jx[a] - cx0];
      sy += wy[b] * sx;
    }
    py[p] = sy;
  }
  for (int k = 0; k < PZ; ++k) {
    const int i2 = z0 + k;
    if (i2 >= F.n2) break;
    int jz[2];
    T wz[2];
    prolong_taps<T>(X, 2, i2, F.n2, jz, wz);
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (wz[c] == T(0)) continue;
      s += wz[c] * py[jz[c] - cz0];
    }
    const unsigned i = (unsigned)(i0 + F.n0 * (i1 + F.n1 * i2));
    F.u[i] += s;
  }
}

// the tiles pay off on big 3-d levels
inline bool tiled_transfer(int dim, int fn0, int fn1, int fn2) {
  return dim == 3 && fn2 >= 4 && fn1 >= 4 && (long long)fn0 * fn1 * fn2 >= (1LL << 15);
}

__host__ __device__ inline bool nested_levels(int fn0, int fn1, int fn2, int cn0, int cn1, int cn2) {
  const int f[3] = {fn0, fn1, fn2}, c[3] = {cn0, cn1, cn2};
  for (int a = 0; a < 3; ++a)
    if (!(f[a] == 2 * c[a] || (f[a] == 1 && c[a] == 1))) return false;
  return true;
}

// ---------------------------------------------------------------------------
// The coarse tail: the whole V-cycle from level l0 down to the coarsest level
// in one thread block (levels small enough that launch latency would dominate
// a kernel per stage).  Same arithmetic as the grid kernels, phase by phase,
// separated by block barriers.
// ---------------------------------------------------------------------------
// The cycle's loops run over a "team" of threads: one thread block (the
// coarse tail, the batched columns, the single-block step) or every thread of
// a cooperative grid (the coarse levels of a big grid: no launch per stage).
// rank/size index the team's threads, sync() is its barrier, max() its
// max-reduction (every thread gets the result).
struct BlockTeam {
  __device__ unsigned rank() const { return threadIdx.x; }
  __device__ unsigned size() const { return blockDim.x; }
  __device__ void sync() const { __syncthreads(); }
  __device__ unsigned long long max(unsigned long long v, unsigned long long* sm) const { return block_max(v, sm); }
};

// (three global slots rotate: the slot zeroed at one reduction was last read
// two reductions earlier, with a grid barrier in between)
struct GridTeam {
  unsigned long long* slots;
  int round;
  __device__ unsigned rank() const { return blockIdx.x * blockDim.x + threadIdx.x; }
  __device__ unsigned size() const { return gridDim.x * blockDim.x; }
  __device__ void sync() const { cooperative_groups::this_grid().sync(); }
  __device__ unsigned long long max(unsigned long long v, unsigned long long* sm) {
    v = block_max(v, sm);
    unsigned long long* s = slots + round % 3;
    if (threadIdx.x == 0) atomicMax(s, v);
    if (rank() == 0) slots[(round + 1) % 3] = 0ull;
    sync();
    const unsigned long long r = *(volatile unsigned long long*)s;
    ++round;
    return r;
  }
};

// one NGS sweep of a level by a team: red then black half-sweeps (ordering
// 1), or the lexicographic order hyperplane by hyperplane (0)
template <typename T, int FORM, int MODEL, typename TM = BlockTeam>
__device__ __forceinline__ void block_sweep(const Level<T>& L, const Phys<T>& P, int ordering = 1, TM tm = TM{}) {
  if (ordering == 0) {
    const int nplanes = L.n0 + L.n1 + L.n2 - 2;
    const int nrows = L.n1 * L.n2;
    for (int s = 0; s < nplanes; ++s) {
      for (int t = tm.rank(); t < nrows; t += tm.size()) {
        const int i1 = t % L.n1, i2 = t / L.n1;
        const int i0 = s - i1 - i2;
        if (i0 >= 0 && i0 < L.n0)
          point_update<T, FORM, MODEL>(L, P, (unsigned)(i0 + L.n0 * t), i0, i1, i2);
      }
      tm.sync();
    }
    return;
  }
  const long long nh = (long long)((L.n0 + 1) >> 1) * L.n1 * L.n2;
  for (int color = 0; color < 2; ++color) {
    for (long long t = tm.rank(); t < nh; t += tm.size()) {
      int i0, i1, i2;
      long long i;
      if (color_cell(L.n0, L.n1, t, color, i0, i1, i2, i)) point_update<T, FORM, MODEL>(L, P, i, i0, i1, i2);
    }
    tm.sync();
  }
}

template <typename T, int FORM, int MODEL, typename TM = BlockTeam>
__device__ __forceinline__ T block_defect_norm(const Level<T>& L, const Phys<T>& P, unsigned long long* sm,
                                               TM* tmp = nullptr) {
  TM local{};
  TM& tm = tmp ? *tmp : local;
  unsigned long long mx = 0;
  for (long long i = tm.rank(); i < L.ncell; i += tm.size()) {
    int i0, i1, i2;
    cell_coords(L.n0, L.n1, i, i0, i1, i2);
    const T di = L.g[pix(L, i, i0, i1, i2)] - apply_N<T, FORM, MODEL>(L, P, L.u, i, i0, i1, i2);
    const unsigned long long b = nbits(di);
    mx = b > mx ? b : mx;
  }
  return from_bits<T>(tm.max(mx, sm));
}

// Levels l0..nl-1 of one multigrid cycle by one team, with the recursion of
// Section 3.2 unrolled: pre-smoothing, defect, restriction and the FAS right
// side on the way down; gamma visits of each coarser level (1: V-cycle, 2:
// W-cycle); the coarsest level sweeps until its defect drops by crtol or
// cmax sweeps are done; prolongation and post-smoothing on the way up.  LV
// gives the level views (L(l)) and the transfers from level l:
// restrict(l, fine array, coarse coords) and prolong(l, fine coords).
// (handoff < nl, grid teams only: from level handoff on, block 0 alone runs
// the rest of the cycle with block barriers, as the single-block tail does,
// while the other blocks wait at the next grid barrier; tail_lv gives that
// part's levels and transfers)
template <typename T, int FORM, int MODEL>
struct NoTail {};

template <typename T, int FORM, int MODEL, typename LV, typename TM = BlockTeam, typename TLV = NoTail<T, FORM, MODEL>>
__device__ __forceinline__ void block_cycle(const LV& lv, int l0, int nl, const Phys<T>& P, int nu1, int nu2, int cmax, T crtol,
                            int gamma, int gamma_levels, unsigned long long* sm, unsigned long long& updates,
                            int ordering = 1, TM* tmp = nullptr, int handoff = 1 << 30,
                            const TLV* tail_lv = nullptr) {
  TM local{};
  TM& tm = tmp ? *tmp : local;
  int visits[24];
  int l = l0;
  bool down = true;
  for (;;) {
    if (down) {
      if constexpr (!std::is_same<TLV, NoTail<T, FORM, MODEL>>::value) {
        if (l == handoff) {
          if (blockIdx.x == 0)
            block_cycle<T, FORM, MODEL, TLV>(*tail_lv, l, nl, P, nu1, nu2, cmax, crtol, gamma, gamma_levels, sm,
                                             updates, ordering);
          tm.sync();
          down = false;
          continue;
        }
      }
      if (l == nl - 1) {
        const Level<T>& C = lv.L(l);
        const T d0 = block_defect_norm<T, FORM, MODEL, TM>(C, P, sm, &tm);
        for (int s = 0; s < cmax; ++s) {
          block_sweep<T, FORM, MODEL, TM>(C, P, ordering, tm);
          updates += C.ncell;
          const T dn = block_defect_norm<T, FORM, MODEL, TM>(C, P, sm, &tm);
          if (!(dn > crtol * d0)) break;
        }
        down = false;
        continue;
      }
      const Level<T>& F = lv.L(l);
      for (int s = 0; s < nu1; ++s) block_sweep<T, FORM, MODEL, TM>(F, P, ordering, tm);
      updates += (unsigned long long)nu1 * F.ncell;
      for (long long i = tm.rank(); i < F.ncell; i += tm.size()) {
        int i0, i1, i2;
        cell_coords(F.n0, F.n1, i, i0, i1, i2);
        F.d[i] = F.g[pix(F, i, i0, i1, i2)] - apply_N<T, FORM, MODEL>(F, P, F.u, i, i0, i1, i2);
      }
      tm.sync();
      const Level<T>& C = lv.L(l + 1);
      for (long long J = tm.rank(); J < C.ncell; J += tm.size()) {
        int J0, J1, J2;
        cell_coords(C.n0, C.n1, J, J0, J1, J2);
        lv.restrict2(l, F.u, F.d, J0, J1, J2, C.ubar[J], C.d[J]);
      }
      tm.sync();
      for (long long J = tm.rank(); J < C.ncell; J += tm.size()) {
        int J0, J1, J2;
        cell_coords(C.n0, C.n1, J, J0, J1, J2);
        C.g[J] = apply_N<T, FORM, MODEL>(C, P, C.ubar, J, J0, J1, J2) + C.d[J];
        C.u[J] = C.ubar[J];
      }
      tm.sync();
      visits[l] = 0;
      ++l;
      continue;
    }
    // level l is finished: back to its parent
    if (l == l0) break;
    const int pl = l - 1;
    const int g = (gamma_levels <= 0 || pl < gamma_levels) ? gamma : 1;
    if (++visits[pl] < g) {           // visit the coarser level again (same right side)
      l = pl + 1;
      down = true;
      continue;
    }
    const Level<T>& F = lv.L(pl);
    for (long long i = tm.rank(); i < F.ncell; i += tm.size()) {
      int i0, i1, i2;
      cell_coords(F.n0, F.n1, i, i0, i1, i2);
      F.u[i] += lv.prolong(pl, i0, i1, i2);
    }
    tm.sync();
    for (int s = 0; s < nu2; ++s) block_sweep<T, FORM, MODEL, TM>(F, P, ordering, tm);
    updates += (unsigned long long)nu2 * F.ncell;
    l = pl;
  }
}

template <typename T>
struct DeviceLevels {
  const Level<T>* Ls;
  const Xfer<T>* Xs;
  __device__ const Level<T>& L(int l) const { return Ls[l]; }
  __device__ T restrict(int l, const T* fine, int J0, int J1, int J2) const {
    return restrict_at(Ls[l], Xs[l], fine, J0, J1, J2);
  }
  __device__ void restrict2(int l, const T* fa, const T* fb, int J0, int J1, int J2, T& a, T& b) const {
    a = restrict(l, fa, J0, J1, J2);
    b = restrict(l, fb, J0, J1, J2);
  }
  __device__ T prolong(int l, int i0, int i1, int i2) const { return prolong_at(Ls[l + 1], Xs[l], i0, i1, i2); }
};

template <typename T, int FORM, int MODEL>
__global__ void __launch_bounds__(TAIL_THREADS, 1) k_tail(const Level<T>* __restrict__ Ls, const Xfer<T>* __restrict__ Xs,
                                                       int l0, int nl, Phys<T> P, int nu1, int nu2, int cmax,
                                                       T crtol, int gamma, int gamma_levels, unsigned long long* stats,
                                                       int ordering) {
  __shared__ unsigned long long sm[33];
  unsigned long long updates = 0;
  block_cycle<T, FORM, MODEL>(DeviceLevels<T>{Ls, Xs}, l0, nl, P, nu1, nu2, cmax, crtol, gamma, gamma_levels, sm,
                              updates, ordering);
  if (threadIdx.x == 0 && stats) atomicAdd(stats, updates);
}

// The coarse levels of a big grid as one cooperative launch: block_cycle run
// by every thread of the grid, a grid barrier between phases instead of a
// launch per stage.  Above the single-block tail's first level the transfers
// are the grid kernels' (nested formulas where the levels nest, tables
// otherwise), from it on the tail's (tables): the values equal those of the
// launches it replaces.
template <typename T>
struct CoopLevels {
  const Level<T>* Ls;
  const Xfer<T>* Xs;
  int tail_start;
  __device__ const Level<T>& L(int l) const { return Ls[l]; }
  __device__ bool nested(int l) const {
    const Level<T>& F = Ls[l];
    const Level<T>& C = Ls[l + 1];
    return l < tail_start && nested_levels(F.n0, F.n1, F.n2, C.n0, C.n1, C.n2);
  }
  __device__ T restrict(int l, const T* fine, int J0, int J1, int J2) const {
    return nested(l) ? restrict_nested_at(Ls[l], Ls[l + 1], fine, J0, J1, J2)
                     : restrict_at(Ls[l], Xs[l], fine, J0, J1, J2);
  }
  __device__ void restrict2(int l, const T* fa, const T* fb, int J0, int J1, int J2, T& a, T& b) const {
    a = restrict(l, fa, J0, J1, J2);
    b = restrict(l, fb, J0, J1, J2);
  }
  __device__ T prolong(int l, int i0, int i1, int i2) const {
    return nested(l) ? prolong_nested_at(Ls[l], Ls[l + 1], Xs[l], i0, i1, i2) : prolong_at(Ls[l + 1], Xs[l], i0, i1, i2);
  }
};

// slots: three global words for the grid reductions; stats: the update count
template <typename T, int FORM, int MODEL>
__global__ void __launch_bounds__(COOP_THREADS) k_coop_cycle(const Level<T>* __restrict__ Ls,
                                                             const Xfer<T>* __restrict__ Xs, int l0, int nl,
                                                             int tail_start, Phys<T> P, int nu1, int nu2, int cmax,
                                                             T crtol, int gamma, int gamma_levels,
                                                             unsigned long long* stats, unsigned long long* slots) {
  __shared__ unsigned long long sm[33];
  GridTeam tm{slots, 0};
  if (tm.rank() == 0) slots[0] = slots[1] = slots[2] = 0ull;
  tm.sync();
  unsigned long long updates = 0;
  const DeviceLevels<T> tail{Ls, Xs};
  block_cycle<T, FORM, MODEL, CoopLevels<T>, GridTeam, DeviceLevels<T>>(CoopLevels<T>{Ls, Xs, tail_start}, l0, nl, P,
                                                                        nu1, nu2, cmax, crtol, gamma, gamma_levels,
                                                                        sm, updates, 1, &tm, tail_start, &tail);
  if (tm.rank() == 0 && stats) atomicAdd(stats, updates);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
inline int grid_for(long long n, int bs = 256) {
  long long b = (n + bs - 1) / bs;
  const long long cap = 152LL * 32;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// 3D launch over (units along x, n1 rows, n2 planes): block x-size is a
// power of two between 32 and 128 covering the row
struct Launch3 {
  dim3 grid, block;
};
// (bx_force > 0: that block x-size, as the autotuner chose it)
inline Launch3 launch3(int nx, int n1, int n2, int bx_force = 0) {
  int bx = 32;
  while (bx < nx && bx < 128) bx <<= 1;
  if (bx_force > 0) bx = bx_force;
  Launch3 L;
  L.block = dim3(bx, 1, 1);
  L.grid = dim3((nx + bx - 1) / bx, n1, n2);
  return L;
}

// host: calls fn(LawTag<model>{}) for a runtime law (COMPOSITE included)
template <typename Fn>
inline void by_model(int model, Fn&& fn) {
  if (model == HAVERKAMP) fn(LawTag<HAVERKAMP>{});
  else if (model == GARDNER) fn(LawTag<GARDNER>{});
  else if (model == COMPOSITE) fn(LawTag<COMPOSITE>{});
  else fn(LawTag<VANGENUCHTEN>{});
}

template <typename T, int FORM>
struct Dispatch {
  template <int NK>
  static void sweep_nk(const Level<T>& L, const Phys<T>& P, int model, int color, cudaStream_t s, int bx = 0) {
    const Launch3 g = launch3((L.n0 + 1) >> 1, L.n1, L.n2, bx);
    by_model(model, [&](auto m) {
      k_sweep<T, FORM, decltype(m)::value, NK><<<g.grid, g.block, 0, s>>>(L, P, color);
    });
  }
  // the FP32 increment form compiles the common fixed step counts 1 and 2
  static void sweep(const Level<T>& L, const Phys<T>& P, int model, int color, cudaStream_t s, int bx = 0) {
    if (FORM == FORM_DELTA && P.newton_k == 1) sweep_nk<(FORM == FORM_DELTA ? 1 : 0)>(L, P, model, color, s, bx);
    else if (FORM == FORM_DELTA && P.newton_k == 2)
      sweep_nk<(FORM == FORM_DELTA ? 2 : 0)>(L, P, model, color, s, bx);
    else sweep_nk<0>(L, P, model, color, s, bx);
  }
  template <int ZC, int NK>
  static void sweep_pipe_zk(const Level<T>& L, const Phys<T>& P, int model, int color, cudaStream_t s, int bx) {
    Launch3 g = launch3((L.n0 + 1) >> 1, L.n1, L.n2, bx);
    g.grid.z = (L.n2 + ZC - 1) / ZC;
    by_model(model, [&](auto m) {
      k_sweep_pipe<T, FORM, decltype(m)::value, ZC, NK><<<g.grid, g.block, 0, s>>>(L, P, color, nullptr);
    });
  }
  template <int ZC>
  static void sweep_pipe_z(const Level<T>& L, const Phys<T>& P, int model, int color, cudaStream_t s, int bx) {
    if (FORM == FORM_DELTA && P.newton_k == 1)
      sweep_pipe_zk<ZC, (FORM == FORM_DELTA ? 1 : 0)>(L, P, model, color, s, bx);
    else if (FORM == FORM_DELTA && P.newton_k == 2)
      sweep_pipe_zk<ZC, (FORM == FORM_DELTA ? 2 : 0)>(L, P, model, color, s, bx);
    else sweep_pipe_zk<ZC, 0>(L, P, model, color, s, bx);
  }
  // (levels below 2^20 cells keep one cell per thread unless the autotuner
  // chose otherwise (bx > 0): latency, not load throughput, bounds them.
  // The pipelined kernels take blocks of at most 128 threads.)
  static void sweep_pipe(const Level<T>& L, const Phys<T>& P, int model, int color, int planes, cudaStream_t s,
                         int bx = 0) {
    if (planes <= 1 || L.n2 < 2 || (bx == 0 && L.ncell < (1LL << 20))) sweep(L, P, model, color, s, bx);
    else if (planes == 2) sweep_pipe_z<2>(L, P, model, color, s, bx > 128 ? 128 : bx);
    else if (planes == 4) sweep_pipe_z<4>(L, P, model, color, s, bx > 128 ? 128 : bx);
    else sweep_pipe_z<8>(L, P, model, color, s, bx > 128 ? 128 : bx);
  }
  // one lexicographic sweep: a launch per hyperplane, rows of the plane's
  // i2 range only
  template <int NK>
  static void sweep_lex_nk(const Level<T>& L, const Phys<T>& P, int model, cudaStream_t s) {
    int bx = 32;
    while (bx < L.n1 && bx < 128) bx <<= 1;
    const int nplanes = L.n0 + L.n1 + L.n2 - 2;
    by_model(model, [&](auto m) {
      for (int p = 0; p < nplanes; ++p) {
        const int i2lo = std::max(0, p - (L.n0 - 1) - (L.n1 - 1)), i2hi = std::min(L.n2 - 1, p);
        const dim3 grid((L.n1 + bx - 1) / bx, i2hi - i2lo + 1, 1);
        k_sweep_plane<T, FORM, decltype(m)::value, NK><<<grid, bx, 0, s>>>(L, P, p, i2lo);
      }
    });
  }
  static void sweep_lex(const Level<T>& L, const Phys<T>& P, int model, cudaStream_t s) {
    if (FORM == FORM_DELTA && P.newton_k == 1) sweep_lex_nk<(FORM == FORM_DELTA ? 1 : 0)>(L, P, model, s);
    else if (FORM == FORM_DELTA && P.newton_k == 2) sweep_lex_nk<(FORM == FORM_DELTA ? 2 : 0)>(L, P, model, s);
    else sweep_lex_nk<0>(L, P, model, s);
  }
  // whether sweep_resid applies to a level (the pipelined two-plane kernel)
  static bool fusable(const Level<T>& L, int planes) {
    return FORM == FORM_DELTA && planes == 2 && L.n2 >= 2 && L.ncell >= (1LL << 20);
  }
  // the last half-sweep of a smoothing (colour 1), writing the defects of
  // its cells; residual_color(0) then gives colour 0's: d and ||d||_inf
  // (into *norm) at the end of the smoothing, as one defect pass would
  static void sweep_resid(const Level<T>& L, const Phys<T>& P, int model, unsigned long long* norm, cudaStream_t s) {
    auto sweep_r = [&](auto nk) {
      Launch3 g = launch3((L.n0 + 1) >> 1, L.n1, L.n2);
      g.grid.z = (L.n2 + 1) / 2;
      by_model(model, [&](auto m) {
        k_sweep_pipe<T, FORM, decltype(m)::value, 2, decltype(nk)::value, true><<<g.grid, g.block, 0, s>>>(L, P, 1,
                                                                                                          norm);
      });
    };
    if (FORM == FORM_DELTA && P.newton_k == 1) sweep_r(LawTag<(FORM == FORM_DELTA ? 1 : 0)>{});
    else if (FORM == FORM_DELTA && P.newton_k == 2) sweep_r(LawTag<(FORM == FORM_DELTA ? 2 : 0)>{});
    else sweep_r(LawTag<0>{});
  }
  static void residual_color(const Level<T>& L, const Phys<T>& P, int model, int color, unsigned long long* norm,
                             cudaStream_t s) {
    const Launch3 g = launch3((L.n0 + 1) >> 1, L.n1, L.n2);
    by_model(model, [&](auto m) {
      k_residual_color<T, FORM, decltype(m)::value><<<g.grid, g.block, 0, s>>>(L, P, color, norm);
    });
  }
  static void residual(const Level<T>& L, const Phys<T>& P, int model, unsigned long long* norm,
                       cudaStream_t s, int bx = 0) {
    const Launch3 g = launch3(L.n0, L.n1, L.n2, bx);
    by_model(model, [&](auto m) {
      k_residual<T, FORM, decltype(m)::value><<<g.grid, g.block, 0, s>>>(L, P, norm);
    });
  }
  static void tau(const Level<T>& C, const Phys<T>& P, int model, cudaStream_t s) {
    const Launch3 g = launch3(C.n0, C.n1, C.n2);
    by_model(model, [&](auto m) { k_tau<T, FORM, decltype(m)::value><<<g.grid, g.block, 0, s>>>(C, P); });
  }
  static void restrict2(const Level<T>& F, const Level<T>& C, const Xfer<T>& X, const T* fa, const T* fb,
                        T* ca, T* cb, cudaStream_t s, int cs_mask = 0) {
    const Launch3 g = launch3(C.n0, C.n1, C.n2);
    if (nested_levels(F.n0, F.n1, F.n2, C.n0, C.n1, C.n2))
      k_restrict_nested<T><<<g.grid, g.block, 0, s>>>(F, C, fa, fb, ca, cb, cs_mask);
    else
      k_restrict<T><<<g.grid, g.block, 0, s>>>(F, C, X, fa, fb, ca, cb, cs_mask);
  }
  static void prolong(const Level<T>& F, const Level<T>& C, const Xfer<T>& X, cudaStream_t s) {
    const Launch3 g = launch3(F.n0, F.n1, F.n2);
    if (nested_levels(F.n0, F.n1, F.n2, C.n0, C.n1, C.n2) && tiled_transfer(F.dim, F.n0, F.n1, F.n2)) {
      using TT = TransferTile<T>;
      const dim3 grid((F.n0 + TT::PX - 1) / TT::PX, (F.n1 + TT::PY - 1) / TT::PY, (F.n2 + TT::PZ - 1) / TT::PZ);
      k_prolong_tiled<T><<<grid, TT::PX * TT::PY, 0, s>>>(F, C, X);
    } else if (nested_levels(F.n0, F.n1, F.n2, C.n0, C.n1, C.n2))
      k_prolong_nested<T><<<g.grid, g.block, 0, s>>>(F, C, X);
    else
      k_prolong<T><<<g.grid, g.block, 0, s>>>(F, C, X);
  }
  // the cooperative coarse cycle: the most blocks that can be co-resident
  static int coop_max_blocks(int model) {
    int per_sm = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    by_model(model, [&](auto m) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coop_cycle<T, FORM, decltype(m)::value>, COOP_THREADS,
                                                    0);
    });
    return per_sm * nsm;
  }
  static cudaError_t coop(const Level<T>* dLs, const Xfer<T>* dXs, int l0, int nl, int tail_start, const Phys<T>& P,
                          int model, int nu1, int nu2, int cmax, T crtol, int gamma, int gamma_levels,
                          unsigned long long* stats, unsigned long long* slots, int blocks, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    Phys<T> Pv = P;
    void* args[] = {(void*)&dLs, (void*)&dXs, (void*)&l0, (void*)&nl, (void*)&tail_start, (void*)&Pv, (void*)&nu1,
                    (void*)&nu2, (void*)&cmax, (void*)&crtol, (void*)&gamma, (void*)&gamma_levels, (void*)&stats,
                    (void*)&slots};
    by_model(model, [&](auto m) {
      e = cudaLaunchCooperativeKernel((const void*)k_coop_cycle<T, FORM, decltype(m)::value>, dim3(blocks),
                                      dim3(COOP_THREADS), args, 0, s);
    });
    return e;
  }
  static void tail(const Level<T>* dLs, const Xfer<T>* dXs, int l0, int nl, const Phys<T>& P, int model,
                   int nu1, int nu2, int cmax, T crtol, int gamma, int gamma_levels, unsigned long long* stats,
                   int ordering, cudaStream_t s) {
    by_model(model, [&](auto m) {
      k_tail<T, FORM, decltype(m)::value><<<1, TAIL_THREADS, 0, s>>>(dLs, dXs, l0, nl, P, nu1, nu2, cmax, crtol,
                                                                      gamma, gamma_levels, stats, ordering);
    });
  }
};

}  // namespace rich
