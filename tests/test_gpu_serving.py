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
