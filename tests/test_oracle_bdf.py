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


@pytest.mark.parametrize("lag", [0, 1])
def test_bdf2_lagged_state_of_k_and_xi(lag):
    """The BDF2 state at which K and the xi term are lagged: psi* = 2 psi^n -
    psi^(n-1) (bdf2_lag 0) or psi^n (bdf2_lag 1, the lag of eq. fully-bdf1).
    Every cell's Kc is the law's K at that state, and xi adds xi psi* to g
    (against the same system with xi = 0)."""
    p = W.random_problem(2, (9, 7), W.VANGENUCHTEN, 41, hetero=True, xi=2e-3, scheme=2)
    rng = np.random.default_rng(4)
    psi_n = np.asarray(p["psi0"], dtype=np.float64)
    psi_m = psi_n + rng.uniform(-0.3, 0.3, psi_n.size)

    def prepared(**kw):
        o = Oracle(W.with_opts(p, bdf2_lag=lag, **kw))
        o.set_state(psi_n, psi_m)
        o.prepare(p["dt"], 2)
        return o

    o, o0 = prepared(), prepared(xi=0.0)
    star = o.array(6)
    assert np.array_equal(star, psi_n if lag else 2.0 * psi_n - psi_m)
    assert not np.array_equal(star, 2.0 * psi_n - psi_m if lag else psi_n)
    K = o.Kc(0)
    for i in range(psi_n.size):
        assert K[i] == o.soil(i, star[i])[2], i
    assert np.array_equal(K, o0.Kc(0))
    xi = p["opts"]["xi"]
    assert np.max(np.abs((o.g(0) - o0.g(0)) - xi * star)) <= 1e-15 * np.max(np.abs(o.g(0)))


@pytest.mark.parametrize("max_cycles", [1, 60])
def test_a_step_shifts_the_history_converged_or_not(max_cycles):
    """After a step -- converged, or stopped at the cycle limit (ENOCONV, the
    state then being the last iterate, as the C ABI documents) -- the next
    BDF2 step's history is (the step's result, the state it started from):
    its lagged state is 2 psi^{n+1} - psi^n bit for bit."""
    from oracle.oracle import ORC_ENOCONV
    p = W.random_problem(2, (9, 8), W.GARDNER, 70, scheme=2, tol=1e-14 if max_cycles == 1 else 1e-9,
                         max_cycles=max_cycles)
    o = Oracle(p)
    psi0 = o.state()
    st, info = o.step(p["dt"], 1)
    assert st == (ORC_ENOCONV if max_cycles == 1 else ORC_OK), (st, info)
    psi1 = o.state()
    assert not np.array_equal(psi1, psi0)
    o.prepare(p["dt"], 2)
    assert np.array_equal(o.array(6), 2.0 * psi1 - psi0)
