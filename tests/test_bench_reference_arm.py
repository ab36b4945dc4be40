"""bench.py's reference arm (the CPU oracle) keeps the JSON-line contract; no GPU needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "20",
                           "--steps", "2", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=300)


def test_reference_arm_prints_one_contract_line():
    r = _run()
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    for key in ("metric", "unit", "higher_is_better", "config", "dtype", "data", "ms_per_step"):
        assert key in d
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_serving_rate_sweep_stretches_the_same_requests(monkeypatch):
    """The offered-load sweep serves the reduced trace's own requests, their
    Poisson arrival times scaled by 200/r (exponential gaps at rate 200/s
    become gaps at rate r/s), once per rate, with the FP64 outer layer and
    continuous batching; no GPU call is made (the server is a stand-in)."""
    sys.path.insert(0, ROOT)
    import bench
    seen = []

    def fake_serve(trace, ids, precision, batched):
        seen.append(([p["name"] for p in trace], [p["arrival"] for p in trace], precision, batched))
        return {"completed": len(ids), "makespan_s": 1.0, "solves_per_s": float(len(ids)),
                "cell_updates_per_s": 1.0, "p50_latency_s": 0.1, "p99_latency_s": 0.2}

    monkeypatch.setattr(bench, "_serve", fake_serve)
    out = bench.serving_bench(nreq=12, max_steps=3)
    sweep = out["reduced_mix"]["rate_sweep_batched_mixed_fp64_outer"]
    assert [s["offered_requests_per_s"] for s in sweep] == list(bench.SERVING_RATES)
    base_names, base_arrivals = seen[0][0], seen[0][1]
    runs = seen[len(bench.SERVING_MODES):len(bench.SERVING_MODES) + len(bench.SERVING_RATES)]
    for rate, (names, arrivals, precision, batched) in zip(bench.SERVING_RATES, runs):
        assert names == base_names and precision == 2 and batched
        for a, b in zip(arrivals, base_arrivals):
            assert abs(a - b * 200.0 / rate) <= 1e-12 * max(1.0, a)
