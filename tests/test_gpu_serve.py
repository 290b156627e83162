"""Serving on the GPU: every job's result is the same alone and in a mix of jobs that arrive
while others run (admission by HBM budget, overlapping work on separate streams).

Each job runs on its own handle and stream, so the mix cannot change its arithmetic: results
must agree bit for bit; the bound is 1e-12 (FP64 form)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    from paper_2511_23438_gb300 import inputs, serve
    eng = serve.GpuEngine()
    jobs = inputs.serving_jobs(8, rate=200.0, seed=5, grids=((3, 4), (4, 4), (3, 5)), chis=(16, 32), steps=3,
                               prec="fp64")
    fps = [eng.footprint(j) for j in jobs]
    budget = 3 * max(fps)  # room for about three jobs at a time: the rest queue for memory
    res, st = serve.Server(eng, budget, max_slots=4).run(jobs)
    assert st["completed"] == len(jobs), res
    assert st["peak_budget_in_use"] <= budget
    admits = sorted((r["admit"], r["done"]) for r in res.values())
    assert any(b[0] < a[1] for a, b in zip(admits, admits[1:]))  # overlapping jobs
    for j in jobs:
        alone, _ = serve.Server(eng, budget, max_slots=1).run([dict(j, arrival=0.0)])
        a, m = alone[j["jid"]], res[j["jid"]]
        for k in ("Z", "Z2", "X", "F"):
            assert a[k].shape == (3,)
            assert np.abs(a[k] - m[k]).max() <= 1e-12, (j, k, a[k], m[k])
    print("serve:", {k: st[k] for k in ("jobs_per_s", "latency_p50_s", "latency_p99_s")})
