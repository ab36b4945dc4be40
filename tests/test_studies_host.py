"""Host arithmetic of the temporal-convergence study (Section 4.1) on the CPU:
the reference on twice the cells is brought to the coarse centres by pair
means, errors are max norms, orders are log2 ratios.  The GPU runs are
replaced by synthetic states with a known first-order error."""
import numpy as np

from paper_2606_04292_gb300 import studies


def test_coarsen_is_exact_for_linear_profiles():
    n_ref = 64
    x_ref = (np.arange(n_ref) + 0.5) / n_ref
    x = (np.arange(n_ref // 2) + 0.5) / (n_ref // 2)
    assert np.allclose(studies.coarsen(3.0 - 2.0 * x_ref), 3.0 - 2.0 * x, rtol=0, atol=1e-15)


def test_orders_of_a_first_order_error(monkeypatch):
    n, n_ref = 32, 128
    x = (np.arange(n) + 0.5) / n
    x_ref = (np.arange(n_ref) + 0.5) / n_ref

    def fake_run(nn, tau, times, scheme, tol):
        xx = x if nn == n else x_ref
        states = [(1.0 + 2.0 * xx) * t + (0.0 if nn == n_ref else 0.7 * tau * t * xx) for t in times]
        return states, 0.0, int(round(times[-1] / tau))

    monkeypatch.setattr(studies, "_run_column", fake_run)
    out = studies.temporal_convergence(n=n, n_ref=n_ref, tau0=0.1, ks=range(4), times=(1.0, 2.0), tau_ref=1e-4)
    for t in ("1.0", "2.0"):
        errs = np.array(out["errors"][t])
        # error 0.7 tau t max(x) at the coarse centres, reference brought down twice by pair means
        want = 0.7 * np.array(out["taus"]) * float(t) * x[-1]
        assert np.allclose(errs, want, rtol=1e-12, atol=1e-15)
        assert np.allclose(out["orders"][t], 1.0, atol=1e-12)
    assert out["reference_steps"] == int(round(2.0 / 1e-4))
