"""Request loop for simulation jobs: HBM-budget admission and continuous batching.

A job is one TEBD simulation of the 2D TFIM (grid, chi, initial-state temperature, J, h, dt,
number of Trotter steps, precision form).  Jobs arrive over time; the server admits a job, in
arrival order, when a slot is free and its device footprint (chi^2 d blocks 16 B, the size of
the MPS at full bond dimension) fits what is left of the HBM budget.  Every admitted job keeps
its MPS resident on the device and runs its steps on its own CUDA stream from its own host
thread, so the work of all admitted jobs overlaps on the GPU; the scheduler wakes on every
arrival and every completion, so a job that arrives while others run is admitted as soon as
memory and a slot free up (continuous batching, not a queue in front of one job at a time).
Per job the result is Z_tot, Z_tot^2, X_tot and F_MPS after every step; the server reports
jobs/s and the p50 / p99 time from arrival to result.

Each job's arithmetic runs on its own handle and stream, so its result does not depend on
what else is in the mix.
"""
import collections
import concurrent.futures as cf
import time

import numpy as np


class Job(dict):
    """A job description (see inputs.serving_jobs): jid, arrival, Lx, Ly, chi, dtheta, J, h,
    dt, steps, order, prec, seed."""


class GpuEngine:
    """Runs jobs on one GPU through the C-ABI library (one handle and one stream per job)."""

    def __init__(self, device=0):
        import torch

        from . import build, lib
        build.build()
        lib.load()
        self.lib = lib
        self.torch = torch
        self.device = device

    def footprint(self, job):
        return self.lib.footprint_bytes(self._cfg(job))

    def _cfg(self, job):
        theta = self.lib.initial_theta(job["J"], job["h"], job["dtheta"])
        return self.lib.config(job["Lx"], job["Ly"], job["chi"], theta, prec=job["prec"], J=job["J"], h=job["h"],
                               dt=job["dt"], order=job["order"], seed=job["seed"])

    def run(self, job):
        """All steps of one job; returns {Z, Z2, X, F} arrays over steps."""
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream()
        m = self.lib.MPS(self._cfg(job), stream=stream.cuda_stream)
        out = {k: [] for k in ("Z", "Z2", "X", "F")}
        try:
            for _ in range(job["steps"]):
                m.step(job["J"], job["h"], job["dt"], job["order"], 1)
                o = m.observables()
                out["Z"].append(o["Z"])
                out["Z2"].append(o["Z2"])
                out["X"].append(o["X"])
                out["F"].append(m.fidelity())
            out["truncations"] = m.stats()["truncations"]
        finally:
            m.close()
            stream.synchronize()
        return {k: np.asarray(v) if isinstance(v, list) else v for k, v in out.items()}


class Server:
    """Admission by HBM budget and slots; continuous batching of the admitted jobs."""

    def __init__(self, engine, budget_bytes, max_slots):
        self.engine = engine
        self.budget = int(budget_bytes)
        self.slots = int(max_slots)

    def run(self, jobs, time_scale=1.0):
        """Serve `jobs` (arrival times scaled by time_scale) to completion.

        Returns (results, stats): results[jid] = {Z, Z2, X, F, arrival, admit, done, latency}
        or {error}; stats has jobs/s over the whole run, the service rate over the time the device
        had work (the saturated rate when the offered load exceeds capacity), latency and queue
        wait p50/p99 (s), bond updates/s and the peak budget in use.
        """
        pending = collections.deque(sorted(jobs, key=lambda j: (j["arrival"], j["jid"])))
        running = {}  # future -> (job, footprint, admit time)
        used = 0
        peak = 0
        results = {}
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        with cf.ThreadPoolExecutor(max_workers=max(1, self.slots)) as pool:
            while pending or running:
                # admit, in arrival order, what has arrived and fits
                while pending and pending[0]["arrival"] * time_scale <= now() and len(running) < self.slots:
                    job = pending[0]
                    try:
                        fp = self.engine.footprint(job)
                    except Exception as e:  # an invalid job is reported, the others go on
                        pending.popleft()
                        results[job["jid"]] = {"error": "%s: %s" % (type(e).__name__, e),
                                               "arrival": job["arrival"] * time_scale}
                        continue
                    if fp > self.budget:
                        pending.popleft()
                        results[job["jid"]] = {"error": "footprint %d B exceeds the budget %d B" % (fp, self.budget),
                                               "arrival": job["arrival"] * time_scale}
                        continue
                    if used + fp > self.budget:
                        break
                    pending.popleft()
                    used += fp
                    peak = max(peak, used)
                    running[pool.submit(self.engine.run, job)] = (job, fp, now())
                # wait for a completion or the next arrival
                # (the head job, once arrived, can only be waiting for memory or a slot: wait
                # for a completion; otherwise wake up at its arrival)
                timeout = None
                if pending and pending[0]["arrival"] * time_scale > now():
                    timeout = pending[0]["arrival"] * time_scale - now()
                if not running:
                    time.sleep(timeout or 0.0)
                    continue
                done, _ = cf.wait(list(running), timeout=timeout, return_when=cf.FIRST_COMPLETED)
                for f in done:
                    job, fp, t_admit = running.pop(f)
                    used -= fp
                    t_done = now()
                    arrival = job["arrival"] * time_scale
                    try:
                        r = f.result()
                    except Exception as e:  # a failed job is reported, the others go on
                        r = {"error": "%s: %s" % (type(e).__name__, e)}
                    r.update(arrival=arrival, admit=t_admit, done=t_done, latency=t_done - arrival)
                    results[job["jid"]] = r
        makespan = now()
        ok = [r for r in results.values() if "error" not in r]
        lat = np.array([r["latency"] for r in ok]) if ok else np.zeros(0)
        wait = np.array([r["admit"] - r["arrival"] for r in ok]) if ok else np.zeros(0)
        # time with at least one job on the device: the service rate there is the saturated rate
        busy, end = 0.0, -1.0
        for a, d in sorted((r["admit"], r["done"]) for r in ok):
            if d > end:
                busy += d - max(a, end)
                end = d
        updates = sum(int(r.get("truncations", 0)) for r in ok)
        stats = {"jobs": len(jobs), "completed": len(ok), "failed": len(results) - len(ok), "makespan_s": makespan,
                 "jobs_per_s": len(ok) / makespan if makespan > 0 else 0.0,
                 "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                 "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                 "service_rate_busy_jobs_per_s": len(ok) / busy if busy > 0 else 0.0, "busy_s": busy,
                 "queue_wait_p50_s": float(np.percentile(wait, 50)) if len(wait) else None,
                 "queue_wait_p99_s": float(np.percentile(wait, 99)) if len(wait) else None,
                 "bond_updates_per_s": updates / makespan if makespan > 0 else 0.0,
                 "peak_budget_in_use": peak, "budget": self.budget, "slots": self.slots}
        return results, stats
