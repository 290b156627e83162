"""Serving loop host logic (no GPU): admission by footprint budget and slots, arrival order,
continuous batching, rejection of jobs larger than the budget, latency statistics."""
import math
import threading
import time

import numpy as np

from paper_2511_23438_gb300 import inputs, serve


class FakeEngine:
    """Stands in for the GPU: a job 'runs' for a time proportional to its size and returns
    values derived from its id; records the device memory in use at every moment."""

    def __init__(self):
        self.lock = threading.Lock()
        self.in_use = 0
        self.max_in_use = 0
        self.active = 0
        self.max_active = 0

    def footprint(self, job):
        return job["chi"] ** 2 * 16

    def run(self, job):
        fp = self.footprint(job)
        with self.lock:
            self.in_use += fp
            self.active += 1
            self.max_in_use = max(self.max_in_use, self.in_use)
            self.max_active = max(self.max_active, self.active)
        time.sleep(0.002 * job["steps"] * job["chi"] / 32)
        with self.lock:
            self.in_use -= fp
            self.active -= 1
        k = np.arange(job["steps"])
        return {"Z": job["jid"] + 0.1 * k, "Z2": k * 0.0, "X": k * 0.0, "F": np.ones(job["steps"]),
                "truncations": 10 * job["steps"]}


def _jobs():
    jobs = inputs.serving_jobs(24, rate=400.0, seed=11, grids=((3, 4),), chis=(16, 32, 64), steps=4)
    jobs.append(dict(jobs[0], jid=99, chi=4096, arrival=0.001))  # larger than any budget below
    return jobs


def test_serving_jobs_are_seeded_and_poisson():
    a = inputs.serving_jobs(200, rate=20.0, seed=3)
    b = inputs.serving_jobs(200, rate=20.0, seed=3)
    assert a == b
    gaps = np.diff([j["arrival"] for j in a])
    assert np.all(gaps >= 0) and abs(gaps.mean() - 1 / 20.0) < 0.25 / 20.0
    assert {(j["Lx"], j["Ly"]) for j in a} <= set(inputs.SERVE_GRIDS)
    assert {j["temperature"] for j in a} == {"low", "mid", "high"}


def test_admission_budget_slots_and_order():
    eng = FakeEngine()
    budget = 3 * 64 * 64 * 16
    res, st = serve.Server(eng, budget, max_slots=4).run(_jobs())
    assert eng.max_in_use <= budget and eng.max_active <= 4
    assert st["peak_budget_in_use"] <= budget
    assert "error" in res[99] and "exceeds the budget" in res[99]["error"]
    ok = {j: r for j, r in res.items() if "error" not in r}
    assert len(ok) == 24 and st["completed"] == 24 and st["failed"] == 1
    for j, r in ok.items():
        assert r["admit"] + 1e-9 >= r["arrival"] and r["done"] >= r["admit"]
        assert np.allclose(r["Z"], j + 0.1 * np.arange(4))
    # arrival order is kept at admission
    order = sorted(ok, key=lambda j: (ok[j]["arrival"], j))
    admits = [ok[j]["admit"] for j in order]
    assert all(b + 1e-9 >= a for a, b in zip(admits, admits[1:]))
    # continuous batching: some job is admitted while an earlier-admitted one is still running
    assert any(ok[b]["admit"] < ok[a]["done"] for a, b in zip(order, order[1:]))
    assert st["latency_p50_s"] <= st["latency_p99_s"] and st["jobs_per_s"] > 0


def test_one_slot_serialises():
    eng = FakeEngine()
    res, st = serve.Server(eng, 1 << 40, max_slots=1).run(_jobs()[:6])
    assert eng.max_active == 1 and st["completed"] == 6


class PickyEngine(FakeEngine):
    def footprint(self, job):
        if job["Lx"] > 16:
            raise ValueError("grid must have Lx <= 16")
        return super().footprint(job)


def test_invalid_job_is_reported_and_the_rest_served():
    jobs = _jobs()[:5]
    jobs.append(dict(jobs[0], jid=50, Lx=40, arrival=0.0005))
    res, st = serve.Server(PickyEngine(), 1 << 40, max_slots=2).run(jobs)
    assert "ValueError" in res[50]["error"] and st["completed"] == 5 and st["failed"] == 1


def test_batched_mix_is_seeded():
    a = inputs.batched_mix(64, seed=7)
    assert a == inputs.batched_mix(64, seed=7) and a != inputs.batched_mix(64, seed=8)
    assert all(math.pi / 12 <= j["dtheta"] <= math.pi / 3 for j in a)
    assert {j["chi"] for j in a} <= {32, 64, 128, 256, 512}


def test_busy_time_and_service_rate():
    eng = FakeEngine()
    jobs = [dict(j, arrival=0.0) for j in _jobs()[:8]]  # all at once: the device never idles
    res, st = serve.Server(eng, 1 << 40, max_slots=2).run(jobs)
    assert st["completed"] == 8 and 0 < st["busy_s"] <= st["makespan_s"] + 1e-9
    assert st["service_rate_busy_jobs_per_s"] >= st["jobs_per_s"] - 1e-9
    assert st["queue_wait_p50_s"] <= st["queue_wait_p99_s"] and st["queue_wait_p99_s"] > 0
