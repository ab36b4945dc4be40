"""The paper's temporal-convergence study and Table 3's run on the GPU.

Section 4.1 measures the time discretisation error of the Celia column:
solutions on N = 1024 cells with tau = 0.1 * 2^-k (k = 0..5) at t = 10 s
and t = 50 s, against a reference on N = 2048 cells with tau = 1e-4, in the
discrete max norm; BDF1 shows first order.  ``temporal_convergence`` runs
that study through the batched-column solver (``richards_columns_*``: every
time step of a column inside one launch), one run per CUDA stream and host
thread so that the runs overlap on the device.

The reference lives on twice the cells: a coarse cell centre is the face
between fine cells 2j and 2j + 1, where the linear interpolant of the
reference is the mean of those two values.

``table3_column`` runs Table 3's configuration (the same column on 2048
cells to t = 360 s at tau = 0.1 s, V(5,5)) through the same solver, for its
wall time beside the paper's CPU times.

Command line (prints one JSON object)::

    python -m paper_2606_04292_gb300.studies [--n 1024] [--n-ref 2048] [--tau-ref 1e-4]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import math
import time

import numpy as np

from . import richards as R
from . import workloads as W


def _run_column(n, tau, times, scheme, tol):
    """Celia column on n cells with step tau; the states at each of times."""
    import torch
    stream = torch.cuda.Stream()
    prob = W.celia_1d(n=n, dt=tau, precision=1, tol=tol)
    cols = R.Columns([prob], stream=stream.cuda_stream)
    states, done = [], 0
    t0 = time.perf_counter()
    for t in times:
        k = int(round(t / tau))
        if abs(k * tau - t) > 1e-9 * t:
            raise ValueError(f"t = {t} is not a multiple of tau = {tau}")
        st = cols.run(tau, k - done, scheme)
        stats = cols.stats()
        if st != R.RICH_OK or int(stats["status"][0]) != R.RICH_OK:
            raise R.RichardsError(st, f"column n={n} tau={tau} failed at t={t}: {stats}")
        done = k
        states.append(cols.state())
    wall = time.perf_counter() - t0
    cols.close()
    return states, wall, done


def coarsen(ref):
    """Values at the centres of a grid of half as many cells (means of pairs)."""
    return 0.5 * (ref[0::2] + ref[1::2])


def temporal_convergence(n=1024, n_ref=2048, tau0=0.1, ks=range(6), times=(10.0, 50.0), tau_ref=1e-4,
                         scheme=1, scheme_ref=1, tol=1e-10):
    """Errors max|psi_tau - I psi_ref| at each time for tau = tau0 2^-k, the
    observed orders log2(e_k / e_{k+1}), and the wall time of each run."""
    if n_ref % n:
        raise ValueError("n_ref must be a multiple of n")
    taus = [tau0 * 2.0 ** -k for k in ks]
    jobs = [(n, tau, scheme) for tau in taus] + [(n_ref, tau_ref, scheme_ref)]
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        futs = [ex.submit(_run_column, nn, tau, times, sch, tol) for nn, tau, sch in jobs]
        results = [f.result() for f in futs]
    ref_states, ref_wall, ref_steps = results[-1]
    out = {"n": n, "n_ref": n_ref, "tau_ref": tau_ref, "scheme": scheme, "scheme_ref": scheme_ref, "tol": tol,
           "taus": taus, "reference_steps": ref_steps, "reference_wall_s": ref_wall,
           "wall_s": [r[1] for r in results[:-1]], "errors": {}, "orders": {}}
    for i, t in enumerate(times):
        ref = ref_states[i]
        while len(ref) > n:
            ref = coarsen(ref)
        errs = [float(np.max(np.abs(r[0][i] - ref))) for r in results[:-1]]
        out["errors"][str(t)] = errs
        out["orders"][str(t)] = [math.log2(errs[j] / errs[j + 1]) for j in range(len(errs) - 1)]
    return out


def table3_column(n=2048, tau=0.1, t_end=360.0, nu=5, kappa=0.1):
    """Table 3's configuration (Section 4.1): the Celia column on n cells to
    t_end with step tau and V(nu, nu) cycles, here through the batched-column
    solver (mixed precision, every step in one launch).  Wall time of the
    whole run, last status and cycles per step."""
    import torch
    nsteps = int(round(t_end / tau))
    prob = W.celia_1d(n=n, dt=tau, nsteps=nsteps, nu1=nu, nu2=nu, kappa=kappa, precision=1)
    stream = torch.cuda.Stream()
    cols = R.Columns([prob], stream=stream.cuda_stream)
    threads = cols.autotune(tau, 1)           # block size for this one column (state restored)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = cols.run(tau, nsteps, 1)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    stats = cols.stats()
    out = {"n": n, "tau": tau, "steps": nsteps, "cycle": f"V({nu},{nu})", "threads": threads, "wall_s": wall,
           "status": R.STATUS_NAMES.get(int(stats["status"][0]), str(int(stats["status"][0]))),
           "run_status": R.STATUS_NAMES.get(st, str(st)), "cycles_per_step": float(stats["cycles"][0]) / nsteps,
           "state": cols.state()}
    cols.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--n-ref", type=int, default=2048)
    ap.add_argument("--tau-ref", type=float, default=1e-4)
    ap.add_argument("--kmax", type=int, default=5)
    args = ap.parse_args()
    t0 = time.perf_counter()
    res = temporal_convergence(n=args.n, n_ref=args.n_ref, tau_ref=args.tau_ref, ks=range(args.kmax + 1))
    res["total_wall_s"] = time.perf_counter() - t0
    print(json.dumps(res))


if __name__ == "__main__":
    main()
