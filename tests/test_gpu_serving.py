"""Continuous batching of Richards requests on one GPU (needs a GPU).

Requests of different sizes, dimensions and soils run concurrently, each on
its own stream with its state resident on the device; each result must be
the same alone and in the mix (no reduction mixes requests, so the
arithmetic is the same), within the step tolerance of the parity tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2606_04292_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_04292_gb300 import richards as R  # noqa: E402
from paper_2606_04292_gb300 import serve  # noqa: E402

STEP_RTOL = 1e-10


def request_mix():
    reqs = [
        W.random_problem(2, (33, 40), W.VANGENUCHTEN, 101, hetero=True, sink=True, scheme=2, precision=1),
        W.random_problem(3, (17, 16, 15), W.HAVERKAMP, 102, scheme=2, precision=1),
        W.random_problem(2, (65, 65), W.GARDNER, 103, sink=True, scheme=1, precision=1),
        W.random_problem(3, (24, 20, 18), W.VANGENUCHTEN, 104, hetero=True, scheme=2, precision=0),
        W.strip_2d(n=65, nsteps=4, precision=1),
        W.random_problem(1, 200, W.VANGENUCHTEN, 105, sink=True, scheme=2, precision=1),
    ]
    for k, p in enumerate(reqs):
        p["nsteps"] = 3 + k % 3
        p["arrival"] = 0.0
    return reqs


def solve_alone(prob):
    s = R.Solver(prob)
    for _ in range(prob["nsteps"]):
        st, info = s.step(prob["dt"], prob["scheme"])
        assert st == R.RICH_OK
    out = s.state()
    s.close()
    return out


def test_each_result_same_alone_and_in_the_mix():
    reqs = request_mix()
    alone = [solve_alone(p) for p in reqs]
    budget = sum(serve.request_bytes(p) for p in reqs[:3])    # forces queueing
    srv = serve.Server(budget_bytes=budget, max_active=3, keep_states=True)
    results, summary = srv.run(reqs, realtime=False)
    assert summary["completed"] == len(reqs)
    for r, ref in zip(results, alone):
        assert r["status"] == "OK"
        err = np.max(np.abs(r["state"] - ref)) / np.max(np.abs(ref))
        assert err <= STEP_RTOL, (r["id"], err)
    # the slot limit held: never more than 3 requests between start and end
    spans = [(r["start"], r["end"]) for r in results]
    for t, _ in spans:
        live = sum(1 for a, b in spans if a <= t < b)
        assert live <= 3


def test_large_requests_same_alone_and_in_the_mix():
    """Requests of the served workload's sizes (a 257^2 strip and a 65^3
    drainage) beside small ones: each result the same alone and in the mix."""
    reqs = [
        W.strip_2d(n=257, nsteps=3, precision=1),
        W.drainage_3d(n=65, nsteps=3, precision=1),
        W.drainage_3d(n=65, nsteps=2, precision=2),
        W.random_problem(2, (129, 129), W.GARDNER, 107, sink=True, scheme=2, precision=1),
        W.random_problem(3, (33, 33, 33), W.HAVERKAMP, 108, scheme=2, precision=0),
    ]
    for k, p in enumerate(reqs):
        p["nsteps"] = p.get("nsteps", 3) if k < 3 else 3
        p["arrival"] = 0.0
    alone = [solve_alone(p) for p in reqs]
    srv = serve.Server(max_active=5, keep_states=True)
    results, summary = srv.run(reqs, realtime=False)
    assert summary["completed"] == len(reqs)
    for r, ref in zip(results, alone):
        assert r["status"] == "OK"
        err = np.max(np.abs(r["state"] - ref)) / np.max(np.abs(ref))
        assert err <= STEP_RTOL, (r["id"], err)


def batch_mix():
    """Mixed-mode requests of every law, 1-3 dimensions, both outer layers,
    sinks, BDF1 and BDF2, different sizes and time steps."""
    reqs = [
        W.random_problem(2, (33, 40), W.VANGENUCHTEN, 111, hetero=True, sink=True, scheme=2, precision=1),
        W.random_problem(3, (17, 16, 15), W.HAVERKAMP, 112, scheme=2, precision=2),
        W.random_problem(2, (65, 65), W.GARDNER, 113, sink=True, scheme=1, precision=1),
        W.strip_2d(n=65, nsteps=4, precision=2),
        W.random_problem(1, 200, W.VANGENUCHTEN, 115, sink=True, scheme=2, precision=1),
        W.random_problem(3, (40, 36, 33), W.VANGENUCHTEN, 116, hetero=True, sink=True, scheme=2, precision=2,
                         dt=120.0),
        W.drainage_3d(n=33, precision=2),
    ]
    for k, p in enumerate(reqs):
        p["nsteps"] = 3 + k % 2
        p["arrival"] = 0.0
        p["opts"] = dict(p["opts"], nu1=2, nu2=2, cycle_gamma=1, gamma_levels=0, coarse_max_sweeps=50,
                         coarse_rtol=0.1, inner_cycles=8, max_outer=60)
    return reqs


def test_batched_steps_equal_single_steps():
    """richards_batcher_step advances every context exactly as richards_step
    does: same cycle and outer counts, the same state (1e-10; the kernels
    evaluate the same per-cell expressions)."""
    reqs = batch_mix()
    stream = torch.cuda.Stream()
    batched = [R.Solver(p, stream=stream.cuda_stream) for p in reqs]
    alone = [R.Solver(p) for p in reqs]
    b = R.Batcher(max_contexts=len(reqs), stream=stream.cuda_stream)
    exact = True
    for step in range(3):
        sts, infos = b.step(batched, [p["dt"] for p in reqs], [p["scheme"] for p in reqs])
        for k, p in enumerate(reqs):
            st, info = alone[k].step(p["dt"], p["scheme"], check=False)
            assert sts[k] == st == R.RICH_OK, (k, sts[k], st)
            for key in ("cycles", "outer_iters", "scheme_used", "cell_updates"):
                assert infos[k][key] == info[key], (step, k, key, infos[k][key], info[key])
            got, want = batched[k].state(), alone[k].state()
            exact = exact and np.array_equal(got, want)
            assert np.max(np.abs(got - want)) <= STEP_RTOL * np.max(np.abs(want)), (step, k)
            assert infos[k]["resid"] == pytest.approx(info["resid"], rel=1e-6, abs=1e-15)
    b.close()
    for s in batched + alone:
        s.close()
    print("batched states bit for bit equal:", exact)


def test_continuous_advance_equals_single_steps():
    """richards_batcher_advance: each context takes its own number of steps
    on its own schedule (calls of a few ticks leave contexts mid-step and
    the next call continues them); every state, and the summed cycle and
    outer counts, equal those of richards_step alone (1e-10)."""
    reqs = batch_mix()
    want = [2 + k % 3 for k in range(len(reqs))]
    streams = [torch.cuda.Stream() for _ in reqs]
    batched = [R.Solver(p, stream=s.cuda_stream) for p, s in zip(reqs, streams)]
    alone = [R.Solver(p) for p in reqs]
    ref_cycles, ref_outer = [], []
    for k, p in enumerate(reqs):
        cyc = outer = 0
        for _ in range(want[k]):
            st, info = alone[k].step(p["dt"], p["scheme"], check=False)
            assert st == R.RICH_OK
            cyc += info["cycles"]
            outer += info["outer_iters"]
        ref_cycles.append(cyc)
        ref_outer.append(outer)
    b = R.Batcher(max_contexts=len(reqs))
    left = list(want)
    got_steps = [0] * len(reqs)
    got_cycles = [0] * len(reqs)
    got_outer = [0] * len(reqs)
    calls = 0
    while any(left):
        idx = [k for k in range(len(reqs)) if left[k] > 0]
        new_left, done, sts, infos = b.advance([batched[k] for k in idx], [reqs[k]["dt"] for k in idx],
                                               [reqs[k]["scheme"] for k in idx], [left[k] for k in idx],
                                               max_ticks=3)
        calls += 1
        for j, k in enumerate(idx):
            assert sts[j] == R.RICH_OK, (k, sts[j])
            left[k] = new_left[j]
            got_steps[k] += done[j]
            if done[j]:
                got_cycles[k] += infos[j]["cycles"]
                got_outer[k] += infos[j]["outer_iters"]
        assert calls < 500
    assert calls > 3                                  # calls did return mid-way
    for k in range(len(reqs)):
        assert got_steps[k] == want[k]
        assert (got_cycles[k], got_outer[k]) == (ref_cycles[k], ref_outer[k]), k
        got, ref = batched[k].state(), alone[k].state()
        assert np.max(np.abs(got - ref)) <= STEP_RTOL * np.max(np.abs(ref)), k
    b.close()
    for s in batched + alone:
        s.close()


def test_batcher_runs_big_requests_on_their_own_cycles():
    """A request whose finest level has at least 2^20 cells takes its inner
    cycles through its own cycle graph under the batcher, beside batched small
    ones; every state and count still equals richards_step's."""
    reqs = [W.drainage_3d(n=129, precision=2), W.drainage_3d(n=33, precision=2),
            W.drainage_3d(n=17, precision=1)]        # 2,146,689 cells (one's own cycles), 35,937, 4,913
    streams = [torch.cuda.Stream() for _ in reqs]
    batched = [R.Solver(p, stream=s.cuda_stream) for p, s in zip(reqs, streams)]
    alone = [R.Solver(p) for p in reqs]
    b = R.Batcher(max_contexts=len(reqs))
    for step in range(2):
        sts, infos = b.step(batched, [p["dt"] for p in reqs], [p["scheme"] for p in reqs])
        for k, p in enumerate(reqs):
            st, info = alone[k].step(p["dt"], p["scheme"], check=False)
            assert sts[k] == st == R.RICH_OK, (step, k, sts[k], st)
            for key in ("cycles", "outer_iters", "cell_updates"):
                assert infos[k][key] == info[key], (step, k, key, infos[k][key], info[key])
            got, want = batched[k].state(), alone[k].state()
            assert np.max(np.abs(got - want)) <= STEP_RTOL * np.max(np.abs(want)), (step, k)
    b.close()
    for s in batched + alone:
        s.close()


def test_batched_server_same_alone_and_in_the_mix():
    """Continuous batching (richards_batcher_advance): requests admitted as
    slots free up (3 slots for 7 requests), each result the same as alone."""
    reqs = batch_mix()
    alone = [solve_alone(p) for p in reqs]
    srv = serve.Server(max_active=3, keep_states=True, batched=True)
    results, summary = srv.run(reqs, realtime=False)
    assert summary["completed"] == len(reqs)
    for r, ref in zip(results, alone):
        assert r["status"] == "OK"
        err = np.max(np.abs(r["state"] - ref)) / np.max(np.abs(ref))
        assert err <= STEP_RTOL, (r["id"], err)
    spans = [(r["start"], r["end"]) for r in results]
    for t, _ in spans:
        assert sum(1 for a, b in spans if a <= t < b) <= 3


def test_batcher_rejects_what_it_cannot_batch():
    reqs = batch_mix()[:2]
    b = R.Batcher(max_contexts=2)
    a = R.Solver(reqs[0])
    fp64 = R.Solver(W.with_opts(reqs[1], precision=0))
    other = R.Solver(W.with_opts(reqs[1], nu2=3))
    for pair_ in ([a, fp64], [a, other], [a, a]):
        with pytest.raises(R.RichardsError) as e:
            b.step(pair_, [60.0, 60.0], [1, 1])
        assert e.value.status == R.RICH_EINVAL
    with pytest.raises(R.RichardsError):
        b.step([a, fp64, other], [60.0] * 3, [1] * 3)      # more than the batcher holds
    with pytest.raises(R.RichardsError) as e:
        b.advance([a], [60.0], [1], [-1])
    assert e.value.status == R.RICH_EINVAL
    for s in (a, fp64, other):
        s.close()
    b.close()


def test_admission_rejects_requests_above_budget():
    reqs = request_mix()[:2]
    small = min(serve.request_bytes(p) for p in reqs)
    srv = serve.Server(budget_bytes=small, max_active=4)
    results, summary = srv.run(reqs, realtime=False)
    statuses = sorted(r["status"] for r in results)
    assert statuses.count("OK") >= 1
    assert summary["completed"] + summary["rejected"] == len(reqs)


def test_busy_context_refuses_other_calls():
    prob = W.random_problem(3, (40, 40, 40), W.VANGENUCHTEN, 106, hetero=True, precision=1)
    stream = torch.cuda.Stream()
    s = R.Solver(prob, stream=stream.cuda_stream)
    L = R.lib()
    h = (C.c_void_p * 1)(s.h.value)
    assert L.richards_batch_submit(h, 1, float(prob["dt"]), 20, 1) == R.RICH_OK
    info = R.richards_step_info()
    st = L.richards_step(s.h, float(prob["dt"]), 1, C.byref(info))
    done = (C.c_int * 1)()
    L.richards_batch_poll(h, 1, done, None, None)
    if not done[0]:
        assert st == R.RICH_EBUSY
        assert L.richards_batch_submit(h, 1, 1.0, 1, 1) == R.RICH_EBUSY
    while not done[0]:
        L.richards_batch_poll(h, 1, done, None, None)
    status = (C.c_int * 1)()
    L.richards_batch_poll(h, 1, done, status, None)
    assert status[0] == R.RICH_OK
    s.close()


def test_poisson_trace_reduced():
    trace = W.serving_trace(rate=200.0, seconds=0.2, seed=6, sizes2d=(65, 129), sizes3d=(17, 33),
                            max_requests=10)
    for p in trace:
        p["nsteps"] = min(p["nsteps"], 5)
    srv = serve.Server(max_active=8)
    results, summary = srv.run(trace, realtime=True)
    assert summary["completed"] == len(trace)
    assert np.isfinite(summary["p50_latency_s"]) and summary["p99_latency_s"] >= summary["p50_latency_s"]
