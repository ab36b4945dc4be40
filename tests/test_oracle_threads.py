"""The oracle's red-black sweep on several OpenMP threads is the same sweep.

Cells of one colour never read one another, so sharing them among threads
cannot change any update: the threaded sweep (used to time the oracle on all
host cores) must equal the serial red-black sweep bit for bit, for every law,
a sink, layered soils and odd sizes.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2606_04292_gb300 import workloads as W

CASES = [
    lambda: W.random_problem(3, (17, 12, 9), W.VANGENUCHTEN, 4, hetero=True, sink=True),
    lambda: W.random_problem(2, (23, 18), W.GARDNER, 3, hetero=True,
                             bc_kinds=[W.DIRICHLET, W.NOFLUX, W.FREE_DRAINAGE, W.FLUX]),
    lambda: W.random_problem(1, 64, W.HAVERKAMP, 2, bc_kinds=[W.FREE_DRAINAGE, W.DIRICHLET]),
    lambda: W.celia_composite_1d(n=40),
]


@pytest.mark.parametrize("mk", CASES)
@pytest.mark.parametrize("threads", [1, 2, 3, 0])
def test_threaded_red_black_sweep_equals_serial(mk, threads):
    prob = mk()
    o = Oracle(prob)
    o.prepare(prob["dt"], 1)
    psi = np.array(prob["psi0"], dtype=np.float64)
    for lev in range(o.nlevels):
        x = psi if lev == 0 else o.restrict(psi) if lev == 1 else np.full(o.ncell(lev), -0.5)
        want = o.sweep(x, lev=lev, ordering=1)
        got, used = o.sweep_threads(x, threads, lev=lev)
        assert used >= 1
        assert np.array_equal(got, want), lev
