"""The command-line runner on the GPU: its steps are the library's steps."""
import json

import numpy as np
import pytest

from paper_2606_04292_gb300 import richards as R
from paper_2606_04292_gb300 import run

pytestmark = pytest.mark.gpu


def test_runner_steps_match_the_solver(capsys):
    argv = ["--workload", "drainage", "--n", "24", "--steps", "2", "--psi0", "-0.5",
            "--opt", "precision=0", "--opt", "nu1=2", "--opt", "coarsest_max_n=4"]
    assert run.main(argv) == 0
    rows = [json.loads(l) for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert [r["step"] for r in rows] == [0, 1] and all(r["status"] == "OK" for r in rows)
    prob = run.build_problem(run.parse(argv))
    with R.Solver(prob, stream=0) as s:
        for r in rows:
            st, info = s.step()
            assert st == R.RICH_OK
            assert info["cycles"] == r["cycles"] and info["cell_updates"] == r["cell_updates"]
        assert np.all(np.isfinite(s.state()))


def test_runner_reports_failure_status(capsys):
    # max_cycles = 1 at tol 1e-14 cannot converge: the step reports ENOCONV and the exit status is 1
    argv = ["--workload", "celia", "--n", "64", "--steps", "3", "--opt", "max_cycles=1", "--opt", "tol=1e-14"]
    assert run.main(argv) == 1
    rows = [json.loads(l) for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(rows) == 1 and rows[0]["status"] == "ENOCONV"


def test_runner_batched_workloads(capsys):
    """The columns and served workloads of the runner step every column and
    request to RICH_OK."""
    assert run.main(["--workload", "columns", "--n", "64", "--steps", "2"]) == 0
    rows = [json.loads(l) for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(rows) == 2 and all(r["columns_ok"] and r["cell_updates"] > 0 for r in rows)
    assert run.main(["--workload", "served", "--n", "3", "--steps", "2"]) == 0
    rows = [json.loads(l) for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(rows) == 2 and all(s == "OK" for r in rows for s in r["status"])
