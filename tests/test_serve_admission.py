"""The serving loop's host logic on the CPU: admission in arrival order by
free slot and device-memory budget (sizes from the library's host-only
richards_device_bytes), rejection of requests larger than the budget, slot
and memory release on completion.  The device side (contexts, batch submit
and poll) is replaced by a fake that finishes each request after a number
of polls proportional to its steps."""
import ctypes as C

import numpy as np
import pytest

from paper_2606_04292_gb300 import richards as R
from paper_2606_04292_gb300 import serve
from paper_2606_04292_gb300 import workloads as W

# a serving loop that never admits or never releases a request spins
# forever: fail such a regression instead of hanging the suite
pytestmark = pytest.mark.timeout(120)


class _FakeDevice:
    def __init__(self, real, budget, max_active):
        self.real = real
        self.budget, self.max_active = budget, max_active
        self.next_id = 1
        self.solvers = {}         # handle -> (prob, bytes)
        self.polls = {}
        self.active_bytes = 0
        self.peak_bytes = 0
        self.peak_active = 0
        self.started = []         # arrival order index of each start

    # -- library calls used by serve ----------------------------------------
    def richards_device_bytes(self, *args):
        return self.real.richards_device_bytes(*args)

    def richards_batch_submit(self, handles, n, dt, nsteps, scheme):
        assert n == 1
        h = handles[0]
        prob, need = self.solvers[h]
        self.polls[h] = max(1, nsteps // 5)
        self.active_bytes += need
        self.peak_bytes = max(self.peak_bytes, self.active_bytes)
        self.peak_active = max(self.peak_active, len(self.polls))
        self.started.append(prob["order"])
        return R.RICH_OK

    def richards_batch_poll(self, handles, n, done, status, info):
        h = handles[0]
        self.polls[h] -= 1
        if self.polls[h] <= 0:
            done[0], status[0] = 1, R.RICH_OK
            info[0].cell_updates = 1
            del self.polls[h]
            self.active_bytes -= self.solvers[h][1]
        else:
            done[0] = 0
        return R.RICH_OK


def _fake_solver_class(dev):
    class FakeSolver:
        def __init__(self, prob, stream=None, opts=None):
            self.h = C.c_void_p(dev.next_id)
            dev.next_id += 1
            dev.solvers[self.h.value] = (prob, serve.request_bytes(prob, opts))

        def close(self):
            pass

        def state(self):
            return np.zeros(1)
    return FakeSolver


class _FakeTorch:
    class cuda:
        class Stream:
            cuda_stream = 0


@pytest.mark.parametrize("max_active", [2, 5])
def test_admission_by_slot_and_memory_budget(monkeypatch, max_active):
    trace = W.serving_trace(rate=200.0, seconds=60.0, seed=6, sizes2d=(129, 257), sizes3d=(65,),
                            max_requests=16)
    for k, p in enumerate(trace):
        p["order"] = k
    sizes = [serve.request_bytes(p) for p in trace]
    budget = int(2.5 * np.median(sizes))             # two or three requests at a time, memory permitting
    huge = dict(W.drainage_3d(n=128), arrival=trace[3]["arrival"], order=-1)
    assert serve.request_bytes(huge) > budget
    trace.insert(4, huge)
    dev = _FakeDevice(R.lib(), budget, max_active)
    monkeypatch.setattr(R, "lib", lambda *a, **k: dev)
    monkeypatch.setattr(R, "Solver", _fake_solver_class(dev))
    srv = serve.Server(budget_bytes=budget, max_active=max_active, poll_s=0.0)
    srv.torch = _FakeTorch
    results, summary = srv.run(trace, realtime=False)
    assert summary["completed"] == 16 and summary["rejected"] == 1
    assert [r["status"] for r in results].count("rejected") == 1
    assert results[4]["status"] == "rejected" and results[4]["bytes"] > budget
    assert dev.peak_bytes <= budget and dev.active_bytes == 0 and not dev.polls
    assert dev.peak_active <= max_active
    assert dev.started == sorted(dev.started)        # admitted in arrival order, never overtaken
    assert dev.peak_active >= min(2, max_active)     # requests overlap when they fit


def test_realtime_admission_waits_for_each_arrival(monkeypatch):
    """With realtime=True no request starts before its arrival time (the
    Poisson trace replayed on the wall clock); latency counts from arrival."""
    trace = W.serving_trace(rate=200.0, seconds=60.0, seed=6, sizes2d=(129,), sizes3d=(65,), max_requests=8)
    for k, p in enumerate(trace):
        p["order"] = k
        p["arrival"] = 0.03 * (k + 1)
    budget = 64 * max(serve.request_bytes(p) for p in trace)
    dev = _FakeDevice(R.lib(), budget, 8)
    monkeypatch.setattr(R, "lib", lambda *a, **k: dev)
    monkeypatch.setattr(R, "Solver", _fake_solver_class(dev))
    srv = serve.Server(budget_bytes=budget, max_active=8, poll_s=1e-3)
    srv.torch = _FakeTorch
    results, summary = srv.run(trace, realtime=True)
    assert summary["completed"] == 8
    for r in results:
        assert r["start"] >= r["arrival"], r
        assert r["latency"] == pytest.approx(r["end"] - r["arrival"]) and r["queue"] >= 0.0
    assert dev.started == list(range(8))
