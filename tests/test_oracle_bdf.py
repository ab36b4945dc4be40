"""Closed forms of the time discretisations on a single cell.

One cell with no-flux faces has no fluxes and no gravity term, so a step
reduces to the time discretisation of d theta/dt = -S(psi).  On the Feddes
plateau (h3 <= psi <= h2) the sink is a constant S, and the steps are the
textbook formulas exactly:
  BDF1 (eq. fully-bdf1):   theta^{n+1} = theta^n - tau S;
  BDF2 (reading):          theta^{n+1} = (4 theta^n - theta^{n-1}) / 3 - (2 tau / 3) S,
with the first step of a run a BDF1 step.  A wrong history weight, time
coefficient or sink sign moves theta by O(tau S) = O(1e-4) here, against a
solve tolerance of 1e-14.
"""
import numpy as np
import pytest

from oracle.oracle import ORC_OK, Oracle
from paper_2606_04292_gb300 import workloads as W


@pytest.mark.parametrize("model", [W.HAVERKAMP, W.GARDNER, W.VANGENUCHTEN])
def test_single_cell_bdf1_then_bdf2_follow_the_closed_forms(model):
    p = W.random_problem(1, (1,), model, 7, bc_kinds=[W.NOFLUX, W.NOFLUX], sink=True, tol=1e-14,
                         max_cycles=200, dt=10.0, L=0.2)         # the cell lies in the root zone
    p["psi0"] = np.array([-1.0])          # on the plateau [h3, h2] = [-5, -0.25] m
    o = Oracle(p)
    S, dS = o.sink(0, -1.0)
    assert S > 0 and dS == 0.0
    tau = p["dt"]
    th = [o.soil(0, -1.0)[0]]
    for k in range(4):
        st, info = o.step(tau, 2)          # the first step falls back to BDF1
        assert st == ORC_OK, info
        psi = o.state()[0]
        assert -5.0 < psi < -0.25          # still on the plateau
        th.append(o.soil(0, psi)[0])
        if k == 0:
            want = th[0] - tau * S
        else:
            want = (4.0 * th[-2] - th[-3]) / 3.0 - (2.0 * tau / 3.0) * S
        assert abs(th[-1] - want) <= 1e-13, (k, th[-1], want)
        assert abs(th[-1] - th[-2]) > 1e-6     # the step did move theta


def test_bdf1_run_is_first_order_forward_in_theta():
    """BDF1 throughout: theta falls by exactly tau S per step on the plateau."""
    p = W.random_problem(1, (1,), W.GARDNER, 8, bc_kinds=[W.NOFLUX, W.NOFLUX], sink=True, tol=1e-14,
                         max_cycles=200, dt=10.0, L=0.2)
    p["psi0"] = np.array([-2.0])
    o = Oracle(p)
    S, _ = o.sink(0, -2.0)
    assert S > 0
    th0 = o.soil(0, -2.0)[0]
    for k in range(1, 5):
        assert o.step(p["dt"], 1)[0] == ORC_OK
        assert abs(o.soil(0, o.state()[0])[0] - (th0 - k * p["dt"] * S)) <= 1e-13 * k
