"""Run time steps of a named workload on the GPU and print one JSON line per step.

    python -m paper_2606_04292_gb300.run --workload drainage --n 192 --steps 2 \
        [--psi0 -0.5] [--opt precision=0 --opt nu1=2 ...]

Workloads: ``drainage`` (3-d heterogeneous van Genuchten drainage, n^3),
``strip`` (2-d infiltration strip, n^2), ``gardner`` (2-d Gardner sine
boundary, n^2), ``two_layer`` (2-d two-layer van Genuchten, n^2) and
``celia`` (1-d Haverkamp column, n cells).  ``--psi0`` replaces the initial
state by a uniform head; ``--opt key=value`` overrides a solver option.  The
solver runs on the default stream; each step's status, cycles, outer
corrections, cell updates and wall time are printed.  Exit status is 0 when
every step returned RICH_OK, 1 otherwise.

Two batched workloads: ``columns`` (n root-uptake columns of U{64..1024}
cells, default 4096, one ``richards_columns_run`` call per step) and
``served`` (the first n requests, default 8, of the Poisson serving trace
with 2-d 129^2-257^2 and 3-d 65^3 grids, all advanced by one
``richards_batcher_step`` per step); ``--opt`` applies to every column or
request, ``--psi0`` does not apply.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import richards as R
from . import workloads as W

WORKLOADS = {"drainage": W.drainage_3d, "strip": W.strip_2d, "gardner": W.gardner_2d,
             "two_layer": W.two_layer_2d, "celia": W.celia_1d}


def _value(text):
    for cast in (int, float):
        try:
            return cast(text)
        except ValueError:
            pass
    return None


def parse(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["columns", "served"], default="drainage")
    ap.add_argument("--n", type=int, default=None, help="cells per axis (the workload's default if absent)")
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--psi0", type=float, default=None, help="uniform initial head")
    ap.add_argument("--opt", action="append", default=[], metavar="KEY=VALUE")
    args = ap.parse_args(argv)
    opts = {}
    for item in args.opt:
        key, sep, val = item.partition("=")
        if not sep:
            ap.error(f"--opt {item!r}: expected KEY=VALUE")
        opts[key] = _value(val)
        if opts[key] is None:
            ap.error(f"--opt {item!r}: the value is not a number")
    args.opts = opts
    return args


def build_problem(args):
    unknown = set(args.opts) - set(W.default_opts())
    if unknown:
        raise SystemExit(f"unknown solver options: {sorted(unknown)}")
    kw = dict(args.opts)
    if args.n is not None:
        kw["n"] = args.n
    prob = WORKLOADS[args.workload](**kw)
    if args.psi0 is not None:
        prob["psi0"] = np.full(W.ncells(prob), float(args.psi0))
    return prob


def _batched_opts(args, base):
    unknown = set(args.opts) - set(W.default_opts())
    if unknown:
        raise SystemExit(f"unknown solver options: {sorted(unknown)}")
    return dict(base, **args.opts)


def run_columns(args):
    probs = W.columns(ncol=args.n or 4096)
    for p in probs:
        p["opts"] = _batched_opts(args, p["opts"])
    ok = True
    cols = R.Columns(probs, stream=0)
    try:
        dt, scheme = probs[0]["dt"], probs[0]["scheme"]
        for k in range(args.steps):
            t0 = time.perf_counter()
            st = cols.run(dt, 1, scheme)           # returns after the stream has finished
            wall = time.perf_counter() - t0
            stt = cols.stats()
            good = st == R.RICH_OK and bool(np.all(stt["status"] == R.RICH_OK))
            ok = ok and good
            print(json.dumps({"step": k, "status": R.STATUS_NAMES.get(st, str(st)), "columns_ok": good,
                              "cell_updates": float(np.sum(stt["updates"])), "wall_s": wall}), flush=True)
            if not good:
                break
    finally:
        cols.close()
    return 0 if ok else 1


def run_served(args):
    import torch
    reqs = W.serving_trace(sizes2d=(129, 257), sizes3d=(65,), max_requests=args.n or 8)
    streams = [torch.cuda.Stream() for _ in reqs]        # each request's own work overlaps
    solvers = []
    for p, st in zip(reqs, streams):
        p["opts"] = _batched_opts(args, p["opts"])
        solvers.append(R.Solver(p, stream=st.cuda_stream))
    ok = True
    b = R.Batcher(max_contexts=max(len(solvers), 1), stream=0)
    try:
        for k in range(args.steps):
            t0 = time.perf_counter()
            sts, infos = b.step(solvers, [p["dt"] for p in reqs], [p["scheme"] for p in reqs])
            wall = time.perf_counter() - t0
            ok = ok and all(st == R.RICH_OK for st in sts)
            print(json.dumps({"step": k, "status": [R.STATUS_NAMES.get(st, str(st)) for st in sts],
                              "cycles": [i["cycles"] for i in infos],
                              "cell_updates": sum(i["cell_updates"] for i in infos), "wall_s": wall}),
                  flush=True)
            if not ok:
                break
    finally:
        b.close()
        for s in solvers:
            s.close()
    return 0 if ok else 1


def main(argv=None):
    args = parse(argv)
    if args.workload == "columns":
        return run_columns(args)
    if args.workload == "served":
        return run_served(args)
    prob = build_problem(args)
    ok = True
    with R.Solver(prob, stream=0) as s:
        for k in range(args.steps):
            t0 = time.perf_counter()
            st, info = s.step(check=False)
            wall = time.perf_counter() - t0
            ok = ok and st == R.RICH_OK
            print(json.dumps({"step": k, "status": R.STATUS_NAMES.get(st, str(st)), "cycles": info["cycles"],
                              "outer": info["outer_iters"], "cell_updates": info["cell_updates"],
                              "wall_s": wall}), flush=True)
            if st != R.RICH_OK:
                break
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
