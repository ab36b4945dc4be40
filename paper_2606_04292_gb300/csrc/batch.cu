// Batched stages of the FP32 inner cycle for many contexts (served requests)
// at once.  Each block finds its descriptor in the launch's list, rebuilds
// the block coordinates the single-context launch would have given it, and
// runs the same kernel body: a request's arithmetic is the same in the batch
// as alone, and nothing mixes requests (each defect norm goes to its own
// context's slot).
#include "kernels.cuh"

namespace rich {

namespace {

__host__ __device__ inline bool nested3(const Level<float>& F, const Level<float>& C) {
  const int f[3] = {F.n0, F.n1, F.n2}, c[3] = {C.n0, C.n1, C.n2};
  for (int a = 0; a < 3; ++a)
    if (!(f[a] == 2 * c[a] || (f[a] == 1 && c[a] == 1))) return false;
  return true;
}

// the level a stage's grid covers, and the units along its rows
__host__ __device__ inline const Level<float>& stage_level(int op, const BJob32& j) {
  return (op == BOP_RESTRICT || op == BOP_TAU) ? j.C : j.F;
}
__host__ __device__ inline int stage_nx(int op, const Level<float>& L) {
  return op == BOP_SWEEP ? (L.n0 + 1) >> 1 : L.n0;
}

template <int OP, int MODEL, int NK>
__device__ __forceinline__ void batch_stage(const BJob32& J, int color, int with_norm, int bx, int by, int bz) {
  if constexpr (OP == BOP_SWEEP) {
    sweep_body<float, FORM_DELTA, MODEL, NK>(J.F, J.P, color, bx, by, bz);
  } else if constexpr (OP == BOP_RESID) {
    __shared__ unsigned long long sm[33];
    unsigned long long mx = residual_body<float, FORM_DELTA, MODEL>(J.F, J.P, bx, by, bz);
    if (with_norm) {                  // (uniform over the launch)
      mx = block_max(mx, sm);
      if (threadIdx.x == 0) atomicMax(J.norm, mx);
    }
  } else if constexpr (OP == BOP_RESTRICT) {
    if (nested3(J.F, J.C)) restrict_nested_body<float>(J.F, J.C, J.F.u, J.F.d, J.C.ubar, J.C.d, bx, by, bz);
    else restrict_body<float>(J.F, J.C, J.X, J.F.u, J.F.d, J.C.ubar, J.C.d, bx, by, bz);
  } else if constexpr (OP == BOP_TAU) {
    tau_body<float, FORM_DELTA, MODEL>(J.C, J.P, bx, by, bz);
  } else {
    if (nested3(J.F, J.C)) prolong_nested_body<float>(J.F, J.C, J.X, bx, by, bz);
    else prolong_body<float>(J.F, J.C, J.X, bx, by, bz);
  }
}

// (the law branch is uniform over a block: one block serves one descriptor)
template <int OP, int NK>
__global__ void __launch_bounds__(BATCH_THREADS) k_batch32(const BJob32* __restrict__ table,
                                                           const __grid_constant__ BList list, int color,
                                                           int with_norm) {
  int k = 0;
  while (k + 1 < list.n && (int)blockIdx.x >= list.block0[k + 1]) ++k;
  const BJob32& J = table[list.job[k]];
  const Level<float>& L = stage_level(OP, J);
  const int gx = (stage_nx(OP, L) + BATCH_THREADS - 1) / BATCH_THREADS;
  const int local = (int)blockIdx.x - list.block0[k];
  const int bx = local % gx, r = local / gx, by = r % L.n1, bz = r / L.n1;
  switch (J.model) {
    case HAVERKAMP: batch_stage<OP, HAVERKAMP, NK>(J, color, with_norm, bx, by, bz); break;
    case GARDNER: batch_stage<OP, GARDNER, NK>(J, color, with_norm, bx, by, bz); break;
    case COMPOSITE: batch_stage<OP, COMPOSITE, NK>(J, color, with_norm, bx, by, bz); break;
    default: batch_stage<OP, VANGENUCHTEN, NK>(J, color, with_norm, bx, by, bz); break;
  }
}

__global__ void __launch_bounds__(TAIL_THREADS, 1) k_tail_batch32(const BJob32* __restrict__ table,
                                                                 const __grid_constant__ BList list, int nu1,
                                                                 int nu2, int cmax, float crtol, int gamma,
                                                                 int gamma_levels) {
  __shared__ unsigned long long sm[33];
  const BJob32& J = table[list.job[blockIdx.x]];
  unsigned long long updates = 0;
  const DeviceLevels<float> lv{J.dLs, J.dXs};
  switch (J.model) {
    case HAVERKAMP:
      block_cycle<float, FORM_DELTA, HAVERKAMP>(lv, J.level, J.nlev, J.P, nu1, nu2, cmax, crtol, gamma,
                                                gamma_levels, sm, updates, 1);
      break;
    case GARDNER:
      block_cycle<float, FORM_DELTA, GARDNER>(lv, J.level, J.nlev, J.P, nu1, nu2, cmax, crtol, gamma,
                                              gamma_levels, sm, updates, 1);
      break;
    case COMPOSITE:
      block_cycle<float, FORM_DELTA, COMPOSITE>(lv, J.level, J.nlev, J.P, nu1, nu2, cmax, crtol, gamma,
                                                gamma_levels, sm, updates, 1);
      break;
    default:
      block_cycle<float, FORM_DELTA, VANGENUCHTEN>(lv, J.level, J.nlev, J.P, nu1, nu2, cmax, crtol, gamma,
                                                   gamma_levels, sm, updates, 1);
      break;
  }
  if (threadIdx.x == 0 && J.stats) atomicAdd(J.stats, updates);
}

template <int OP, int NK>
void launch_op(const BJob32* table, const BList& list, int color, bool with_norm, cudaStream_t s) {
  const int blocks = list.block0[list.n];
  if (blocks <= 0) return;
  k_batch32<OP, NK><<<blocks, BATCH_THREADS, 0, s>>>(table, list, color, with_norm ? 1 : 0);
}

template <int OP>
void launch_nk(int nk, const BJob32* table, const BList& list, int color, bool with_norm, cudaStream_t s) {
  if (OP != BOP_SWEEP || nk == 0) launch_op<OP, 0>(table, list, color, with_norm, s);
  else if (nk == 1) launch_op<OP, 1>(table, list, color, with_norm, s);
  else launch_op<OP, 2>(table, list, color, with_norm, s);
}

}  // namespace

int batch_blocks(int op, const BJob32& j) {
  const Level<float>& L = stage_level(op, j);
  const long long gx = (stage_nx(op, L) + BATCH_THREADS - 1) / BATCH_THREADS;
  return (int)(gx * L.n1 * L.n2);
}

void batch32(int op, int nk, const BJob32* table, const BList& list, int color, bool with_norm, cudaStream_t s) {
  switch (op) {
    case BOP_SWEEP: launch_nk<BOP_SWEEP>(nk, table, list, color, with_norm, s); break;
    case BOP_RESID: launch_nk<BOP_RESID>(nk, table, list, color, with_norm, s); break;
    case BOP_RESTRICT: launch_nk<BOP_RESTRICT>(nk, table, list, color, with_norm, s); break;
    case BOP_TAU: launch_nk<BOP_TAU>(nk, table, list, color, with_norm, s); break;
    default: launch_nk<BOP_PROLONG>(nk, table, list, color, with_norm, s); break;
  }
}

void batch_tail32(const BJob32* table, const BList& list, int nu1, int nu2, int cmax, float crtol, int gamma,
                  int gamma_levels, cudaStream_t s) {
  if (list.n <= 0) return;
  k_tail_batch32<<<list.n, TAIL_THREADS, 0, s>>>(table, list, nu1, nu2, cmax, crtol, gamma, gamma_levels);
}

}  // namespace rich
