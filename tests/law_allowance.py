"""Law-error allowance for comparing a mixed-precision result with the oracle.

The mixed mode evaluates K(psi*), theta and its defect in float-float
arithmetic, within a relative error eps of FP64.  Its discrete system then
differs from the oracle's by at most eps times the size of each term of
g - N(psi) that depends on K or theta, so the oracle's FP64 residual of a
mixed result may exceed the GPU's own by that much.  law_allowance returns
eps times, per cell, the magnitudes of those terms (interior fluxes
|m_f (psi_i - psi_j)|, Dirichlet diagonals, gravity fluxes, |g|, a theta_s,
the sink coefficient), maximised over cells, in theta units (divided by a).
"""
import numpy as np


def law_allowance(orc, prob, psi, eps):
    n0, n1, n2 = prob["n"]
    dim = prob["dim"]
    Kc = orc.Kc(0).reshape(n2, n1, n0)
    P = np.asarray(psi, dtype=np.float64).reshape(n2, n1, n0)
    h = [prob["L"][a] / prob["n"][a] for a in range(dim)]
    mats = prob["soil"].get("materials")
    ts = max(m["theta_s"] for m in mats) if mats else prob["soil"]["theta_s"]
    tot = np.abs(orc.g(0)).reshape(n2, n1, n0) + orc.a * ts
    for a in range(dim):
        ax = 2 - a
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[ax], sl_hi[ax] = slice(0, -1), slice(1, None)
        Kf = 0.5 * (Kc[tuple(sl_lo)] + Kc[tuple(sl_hi)])
        flux = Kf / h[a] ** 2 * np.abs(P[tuple(sl_hi)] - P[tuple(sl_lo)])
        if a == dim - 1:
            flux = flux + Kf / h[a]                     # gravity
        tot[tuple(sl_lo)] += flux
        tot[tuple(sl_hi)] += flux
        for side in range(2):
            kb = orc.array(10 + 2 * a + side, 0)
            edge = [slice(None)] * 3
            edge[ax] = -1 if side else 0
            bval = abs(prob["bc"]["value"][2 * a + side])
            tot[tuple(edge)] += 2.0 * kb.reshape(tot[tuple(edge)].shape) / h[a] ** 2 * (np.abs(P[tuple(edge)]) + bval)
    if prob["sink"]["enabled"]:
        tot += orc.array(4, 0).reshape(n2, n1, n0)
    return eps * float(np.max(tot)) / orc.a
