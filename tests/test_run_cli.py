"""The command-line runner's argument handling (no GPU: problems are only built)."""
import numpy as np
import pytest

from paper_2606_04292_gb300 import run
from paper_2606_04292_gb300 import workloads as W


def test_options_and_uniform_state():
    a = run.parse(["--workload", "drainage", "--n", "16", "--psi0", "-0.5",
                   "--opt", "precision=0", "--opt", "nu1=2", "--opt", "tol=1e-9"])
    p = run.build_problem(a)
    assert p["n"] == (16, 16, 16)
    assert p["opts"]["precision"] == 0 and p["opts"]["nu1"] == 2 and p["opts"]["tol"] == 1e-9
    assert isinstance(p["opts"]["nu1"], int)
    assert np.array_equal(p["psi0"], np.full(16 ** 3, -0.5))
    # the workload's own options stay where not overridden
    assert p["opts"]["cycle_gamma"] == W.drainage_3d(n=16)["opts"]["cycle_gamma"]


@pytest.mark.parametrize("name", sorted(run.WORKLOADS))
def test_every_workload_builds(name):
    n = {"celia": 32}.get(name, 16)
    p = run.build_problem(run.parse(["--workload", name, "--n", str(n)]))
    assert W.ncells(p) == n ** p["dim"]


def test_rejects_unknown_option_and_malformed_pairs():
    with pytest.raises(SystemExit):
        run.build_problem(run.parse(["--opt", "bogus=1"]))
    with pytest.raises(SystemExit):
        run.parse(["--opt", "nu1"])
    with pytest.raises(SystemExit):
        run.parse(["--opt", "nu1=two"])
