"""Brute-force solve of one implicit step -- TEST INFRASTRUCTURE ONLY.

Solves N_h(psi) = g_h (eq. Nh-def) on a tiny grid by Newton's method on the
full system with a dense Jacobian J = diag(a theta' + S' + xi) + M and a
library linear solve (numpy.linalg.solve), with step halving on the residual
max norm.  This is the plain definition of the step's result, independent of
the NGS smoother, the FAS hierarchy and the transfer operators.
"""
import numpy as np


def dense_newton(orc, psi0, tol=1e-14, maxit=100):
    """Return psi with ||g - N(psi)||_inf * tau_eff <= tol (after orc.prepare)."""
    a = orc.a
    xi = orc.prob["opts"]["xi"]
    M = orc.dense_M(0)
    g = orc.g(0)
    psi = np.array(psi0, dtype=np.float64)
    r, nrm = orc.residual(psi, g)
    for _ in range(maxit):
        if nrm / a <= tol:
            break
        d = np.empty_like(psi)
        for i in range(len(psi)):
            _, dth, _ = orc.soil(i, psi[i])
            _, dS = orc.sink(i, psi[i])
            d[i] = a * dth + dS + xi
        J = M + np.diag(d)
        step = np.linalg.solve(J, r)          # J dpsi = g - N(psi)
        lam = 1.0
        while lam > 1e-6:
            trial = psi + lam * step
            rt, nt = orc.residual(trial, g)
            if nt < nrm or nt / a <= tol:
                break
            lam *= 0.5
        psi, r, nrm = trial, rt, nt
    return psi, nrm / a
