// Host-side checks of the physical inputs (Table 1's laws, the sink reading
// of assumption (A2), boundary conditions), shared by every entry point that
// accepts them so that all of them reject the same inputs.  Each returns
// nullptr when the input is valid, else a short complaint.
#pragma once
#include <cmath>

#include "richards.h"

namespace rich {

// One law's parameters; p1/p2 given by per-cell fields are checked separately.
inline const char* law_error(int model, double Ks, double ts, double tr, double p1, double p2, double p3, double p4,
                             bool p1_field, bool p2_field) {
  const bool ok = model >= 0 && model <= 2 && std::isfinite(Ks) && Ks > 0.0 && std::isfinite(ts) &&
                  std::isfinite(tr) && tr >= 0.0 && ts > tr;
  if (!ok) return "invalid soil: need a known law, Ks > 0, theta_s > theta_r >= 0";
  auto pos = [](double x) { return std::isfinite(x) && x > 0.0; };
  if (model == RICH_HAVERKAMP && !(pos(p3) && pos(p4) && (p1_field || pos(p1)) && (p2_field || pos(p2))))
    return "Haverkamp needs alpha, beta, A, gamma > 0";
  if (model == RICH_GARDNER && !(p1_field || pos(p1))) return "Gardner needs alpha > 0";
  if (model == RICH_VANGENUCHTEN &&
      !((p1_field || pos(p1)) && (p2_field || (std::isfinite(p2) && p2 > 1.0)) && std::isfinite(p3)))
    return "van Genuchten needs alpha > 0, n > 1, finite l";
  return nullptr;
}

// The sink's parameters (only when it is enabled).
inline const char* sink_error(const richards_sink& k) {
  if (!k.enabled) return nullptr;
  const double v[] = {k.Tp, k.root_depth, k.root_decay, k.h1, k.h2, k.h3, k.h4};
  for (double x : v)
    if (!std::isfinite(x)) return "non-finite sink parameter";
  if (!(k.h4 < k.h3 && k.h3 <= k.h2 && k.h2 < k.h1) || !(k.Tp >= 0.0) || !(k.root_decay > 0.0) ||
      !(k.root_depth > 0.0))
    return "sink needs h4 < h3 <= h2 < h1, Tp >= 0, root depth and decay > 0";
  return nullptr;
}

// Boundary kinds and scalar values of the 2*dim faces (value fields are
// checked by the caller where it can read them).
inline const char* bc_error(const richards_bc& b, int dim) {
  for (int f = 0; f < 2 * dim; ++f) {
    if (b.kind[f] < 0 || b.kind[f] > 3) return "unknown boundary kind";
    if (b.kind[f] == RICH_BC_FREE_DRAINAGE && f != 2 * (dim - 1))
      return "free drainage is only defined on the bottom face";
    if (!std::isfinite(b.value[f])) return "non-finite boundary value";
  }
  return nullptr;
}

}  // namespace rich
