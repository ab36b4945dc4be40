// FP32 instantiations: the inner correction problem of the mixed mode (the
// half-sweeps are in k32s.cu).
#include "kernels.cuh"

namespace rich {
using D = Dispatch<float, FORM_DELTA>;
void residual32(const Level<float>& L, const Phys<float>& P, int model, unsigned long long* norm,
                cudaStream_t s, int bx) {
  D::residual(L, P, model, norm, s, bx);
}
void tau32(const Level<float>& C, const Phys<float>& P, int model, cudaStream_t s) { D::tau(C, P, model, s); }
void restrict32(const Level<float>& F, const Level<float>& C, const Xfer<float>& X, const float* fa,
                const float* fb, float* ca, float* cb, cudaStream_t s, int cs_mask) {
  D::restrict2(F, C, X, fa, fb, ca, cb, s, cs_mask);
}
void prolong32(const Level<float>& F, const Level<float>& C, const Xfer<float>& X, cudaStream_t s) {
  D::prolong(F, C, X, s);
}
void tail32(const Level<float>* dLs, const Xfer<float>* dXs, int l0, int nl, const Phys<float>& P, int model,
            int nu1, int nu2, int cmax, float crtol, int gamma, int gamma_levels, unsigned long long* stats,
            int ordering, cudaStream_t s) {
  D::tail(dLs, dXs, l0, nl, P, model, nu1, nu2, cmax, crtol, gamma, gamma_levels, stats, ordering, s);
}
int coop_max_blocks32(int model) { return D::coop_max_blocks(model); }
cudaError_t coop32(const Level<float>* dLs, const Xfer<float>* dXs, int l0, int nl, int tail_start,
                   const Phys<float>& P, int model, int nu1, int nu2, int cmax, float crtol, int gamma,
                   int gamma_levels, unsigned long long* stats, unsigned long long* slots, int blocks,
                   cudaStream_t s) {
  return D::coop(dLs, dXs, l0, nl, tail_start, P, model, nu1, nu2, cmax, crtol, gamma, gamma_levels, stats, slots,
                 blocks, s);
}
void residual_color32(const Level<float>& L, const Phys<float>& P, int model, int color, unsigned long long* norm,
                      cudaStream_t s) {
  D::residual_color(L, P, model, color, norm, s);
}
}  // namespace rich
