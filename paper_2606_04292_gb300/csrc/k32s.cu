// FP32 instantiations, second unit: the half-sweeps of the inner correction
// problem (the largest kernels; compiled beside k32.cu).
#include "kernels.cuh"

namespace rich {
using D = Dispatch<float, FORM_DELTA>;
void sweep32(const Level<float>& L, const Phys<float>& P, int model, int color, int planes, cudaStream_t s,
             int bx) {
  D::sweep_pipe(L, P, model, color, planes, s, bx);
}
bool resid_fusable32(const Level<float>& L, int planes) { return D::fusable(L, planes); }
void sweep_resid32(const Level<float>& L, const Phys<float>& P, int model, unsigned long long* norm,
                   cudaStream_t s) {
  D::sweep_resid(L, P, model, norm, s);
}
void sweep_lex32(const Level<float>& L, const Phys<float>& P, int model, cudaStream_t s) { D::sweep_lex(L, P, model, s); }
}  // namespace rich
