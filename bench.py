"""Benchmark: bond updates/s of grouped-qubit MPS TEBD on a 6x8 TFIM grid at chi = 1024.

One step = one Trotter step of the whole hot path (in-block X / ZZ layers, every
inter-block ZZ gate as a rank-2 MPO with the truncation of each spanned bond, and
the <Z_tot>, <Z_tot^2>, <X_tot> environment sweep) on a device-resident MPS.
A bond update is one truncation of one bond (172 per step at 6x8).  Warm-up steps
also grow the bonds from the product state to chi.  Inputs larger than L2: the MPS
at chi = 1024 holds ~1.6 GB (complex64) and every step streams all of it.

Multi-GPU: replicas only (one independent MPS per rank, no collective on the data
path); value = bond updates of all ranks / max over ranks of the timed region.

--impl reference times the CPU oracle (oracle/, NumPy FP64) on the host cores on a
bounded sample of the same workload and prints the same JSON line: bond updates at the
identical shape (6x8, every bond at chi = 1024) on a seeded random canonical MPS, one
adjacent inter-block gate (one bond update) per step.

Besides the split-precision form (the timed default), the line reports the FP64 form at the
same shape (a few bond updates of the evolved state, converted to complex128), the serving
loop on a mix drawn like the serving configuration, and per-site device times.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID = (6, 8)
TEMP_DTHETA = 2.0 * math.pi / 9.0  # mid temperature
J, HX, DT, ORDER = -1.0, 2.0, 0.25, 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chi", type=int, default=1024)
    ap.add_argument("--prec", default="split_bf16x3")
    ap.add_argument("--grid", default="%dx%d" % GRID)
    ap.add_argument("--cpu-updates", type=int, default=1, help="oracle bond updates timed for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-updates", type=int, default=2, help="FP64-form bond updates timed at full shape (0: none)")
    ap.add_argument("--other-split", default="split_tf32x3", help="also time one step of this form on the evolved "
                    "state ('' : none)")
    ap.add_argument("--serve-jobs", type=int, default=16, help="jobs of the short serving run (0: none)")
    ap.add_argument("--serve-steps", type=int, default=3, help="Trotter steps per serving job")
    ap.add_argument("--batch-mps", type=int, default=64, help="MPS of the batched-advance leg (0: none)")
    ap.add_argument("--three-d", default="3x3x4", help="open 3D grid of the one-qubit-per-site leg ('' : none)")
    ap.add_argument("--three-d-chi", type=int, default=128)
    ap.add_argument("--xy", default="6x6", help="open grid of the XY-model leg ('' : none)")
    ap.add_argument("--xy-chi", type=int, default=32)
    ap.add_argument("--save-state", default="", help="write the evolved MPS of the timed run to this checkpoint")
    ap.add_argument("--one-gate", default="", help="load this checkpoint, apply one adjacent gate between the "
                    "middle blocks (a single bond-update unit of the step, for launch lists), print it and exit")
    ap.add_argument("--peaks", action="store_true", help="measure dense matmul rates (torch) and exit")
    ap.add_argument("--split-error", default="", help="error table of the complex64 forms against the FP64 GPU "
                    "form: comma-separated chi:steps pairs on the 5x6 grid (e.g. 64:20,256:8), then exit")
    ap.add_argument("--split-perturb", type=float, default=0.0, help="with --split-error: start the compared "
                    "handle at theta + this value (with --prec fp64: the sensitivity floor of the run)")
    return ap.parse_args()


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, dev):
        self.dev, self.samples, self.proc = dev, [], None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def measure_peaks():
    """Dense matmul rates of this GPU through torch (cuBLAS): FP64, FP32 (no TF32), TF32, BF16,
    complex64 and complex128, 8192^3 (4096^3 complex), best of 10 after warm-up, CUDA events."""
    import torch

    out = {}
    for name, dt, nn, tf32 in (("fp64", torch.float64, 8192, False), ("fp32", torch.float32, 8192, False),
                               ("tf32", torch.float32, 8192, True), ("bf16", torch.bfloat16, 8192, False),
                               ("c64", torch.complex64, 4096, False), ("c128", torch.complex128, 4096, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(nn, nn, device="cuda", dtype=dt)
        b = torch.randn(nn, nn, device="cuda", dtype=dt)
        for _ in range(3):
            a @ b
        best = 1e30
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        flops = (8.0 if dt in (torch.complex64, torch.complex128) else 2.0) * nn ** 3
        out[name + "_tflops"] = flops / (best / 1e3) / 1e12
    torch.backends.cuda.matmul.allow_tf32 = False
    out["device"] = torch.cuda.get_device_name()
    return out


def serve_run(njobs, steps, prec):
    """A serving run drawn like the serving configuration: Poisson arrivals (20 jobs/s, seeded),
    grids uniform over 4x4 / 5x6 / 6x6 / 6x8 / 7x8, chi uniform over {64, 256, 1024}, temperature
    uniform over low / mid / high, second-order steps; the HBM budget is the device's free memory
    at the start (less 4 GB of headroom), 8 slots.  Fewer jobs and steps than the configuration's
    200 x 20 keep the run within the benchmark's minutes."""
    import torch
    from paper_2511_23438_gb300 import inputs, serve

    free, _ = torch.cuda.mem_get_info()
    budget = max(1 << 30, free - (4 << 30))
    jobs = inputs.serving_jobs(njobs, rate=20.0, seed=20261203, chis=(64, 256, 1024), steps=steps, prec=prec)
    res, st = serve.Server(serve.GpuEngine(), budget, max_slots=8).run(jobs)
    st["workload"] = ("%d jobs, Poisson 20/s, grids %s, chi {64,256,1024}, temperatures low/mid/high, %d steps "
                      "each, %s, 8 slots, budget %.1f GB (free HBM less 4 GB)"
                      % (njobs, "/".join("%dx%d" % g for g in inputs.SERVE_GRIDS), steps, prec, budget / 1e9))
    return st


# adjacent inter-block gates between the two middle blocks of the chain (every bond around them
# at chi for chi <= 1024 on the 6x8 grid): the bond updates timed for the oracle and the FP64 form;
# `inter` is a gate schedule (p, q, ...) in application order
def middle_adjacent_gates(inter, Lx):
    mid = Lx - 1
    return [i for i, g in enumerate(inter) if g[0] == mid and g[1] == mid + 1]


class OracleSample:
    """The oracle, as it stands, on bond updates at the benchmark's shape: a seeded random
    canonical MPS of the same grid with every bond at min(chi, bound) (the shapes the timed steps
    work on once the bonds have grown), centre on the middle block; each update is one adjacent
    inter-block gate there (rank-2 MPO, LQ of the right block, SVD of the centre block,
    truncation to chi), preceded by the gauge move the previous update left behind."""

    def __init__(self, Lx, Ly, chi):
        from oracle import layout, mps

        t0 = time.perf_counter()
        self.m = mps.random_canonical(Lx, Ly, chi, seed=20261203, decay=chi / 8.0, centre=Lx - 1)
        self.gen_s = time.perf_counter() - t0
        self.inter = layout.schedule(Lx, Ly)[1]
        self.gates = middle_adjacent_gates(self.inter, Lx)
        self.i = 0
        self.Lx, self.Ly, self.chi = Lx, Ly, chi

    def update(self, phi):
        g = self.inter[self.gates[self.i % len(self.gates)]]
        self.i += 1
        n0 = len(self.m.fidelities)
        t0 = time.perf_counter()
        self.m.zz_inter(g, phi)
        return len(self.m.fidelities) - n0, time.perf_counter() - t0

    def describe(self, n, secs):
        return ("oracle (NumPy FP64, LAPACK QR + SVD): %d bond update(s) at the identical shape -- %dx%d grid, "
                "every bond at chi=%d, adjacent gate between the middle blocks (LQ of a 2048 x 16384 block, "
                "SVD of a 16384 x 2048 centre) -- on a seeded random canonical MPS, %.1f s (state generated "
                "untimed in %.1f s)" % (n, self.Lx, self.Ly, self.chi, secs, self.gen_s))


def batched_run(lib, count, prec):
    """The batched workload: `count` independent MPS drawn like the batched configuration (grids
    4x4 .. 6x6, chi uniform over {32, ..., 512}, dtheta uniform in [pi/12, pi/3], seeded), each on
    a CUDA stream of its own and grown by two untimed Trotter steps; then one step of every MPS is
    timed twice: handle after handle on one host thread, and through mpsgb_batch_step (one host
    thread per handle, overlapping on the device, fixed launch sequences replayed as CUDA graphs)."""
    import torch
    from paper_2511_23438_gb300 import inputs

    mix = inputs.batched_mix(count, seed=20261203, prec=prec)
    streams = [torch.cuda.Stream() for _ in mix]
    ms = []
    for j, s in zip(mix, streams):
        th = lib.initial_theta(j["J"], j["h"], j["dtheta"])
        cfg = lib.config(j["Lx"], j["Ly"], j["chi"], th, prec=prec, J=j["J"], h=j["h"], dt=j["dt"], order=j["order"])
        ms.append(lib.MPS(cfg, stream=s.cuda_stream))
    lib.batch_step(ms, 2, use_graph=1)

    def updates():
        return sum(m.stats()["truncations"] for m in ms)

    u0 = updates()
    t0 = time.perf_counter()
    for m in ms:
        m.step(m.cfg.J, m.cfg.h, m.cfg.dt, m.cfg.trotter_order, 1)
        m.observables()
    t_seq = time.perf_counter() - t0
    u1 = updates()
    t0 = time.perf_counter()
    lib.batch_step(ms, 1, use_graph=1)
    for m in ms:
        m.observables()
    t_bat = time.perf_counter() - t0
    u2 = updates()
    for m in ms:
        m.close()
    return {"mps": count, "precision": prec, "sequential_bond_updates_per_s": (u1 - u0) / t_seq,
            "batched_bond_updates_per_s": (u2 - u1) / t_bat, "sequential_s": t_seq, "batched_s": t_bat,
            "bond_updates_per_step": u2 - u1,
            "workload": "%d MPS, grids 4x4..6x6, chi in {32..512}, dtheta in [pi/12, pi/3], one stream each, two "
                        "untimed steps, then one timed step per MPS (wall clock, host-synchronised)" % count}


def three_d_run(lib, dims, chi, prec, grow=2):
    """The 3D variant: an open Lx x Ly x Lz cubic grid, one qubit per MPS site (d = 2) along the 3D
    snake, mid temperature (dtheta = pi/9, theta_min at coordination 6), J = -1, h = 2, dt = 0.25,
    second order; `grow` untimed steps from the product state, then one step timed with CUDA
    events on the handle's stream."""
    import torch
    Lx, Ly, Lz = (int(v) for v in dims.split("x"))
    th = lib.initial_theta(J, HX, math.pi / 9, lattice=lib.LATTICE_3D_SITES)
    s = torch.cuda.Stream()
    m = lib.MPS(lib.config(Lx, Ly, chi, th, prec=prec, J=J, h=HX, dt=DT, order=2, lattice=lib.LATTICE_3D_SITES, Lz=Lz),
                stream=s.cuda_stream)
    m.step(J, HX, DT, 2, grow)
    u0 = m.stats()["truncations"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    m.step(J, HX, DT, 2, 1)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    u = m.stats()["truncations"] - u0
    out = {"workload": "3D TFIM %dx%dx%d open grid, one qubit per site (d=2, %d sites), chi=%d, mid temperature "
                       "(dtheta=pi/9), %d untimed steps then one timed" % (Lx, Ly, Lz, Lx * Ly * Lz, chi, grow),
           "precision": prec, "bond_updates_per_s": u / (ms / 1e3), "ms_per_step": ms, "bond_updates_per_step": u,
           "F": m.fidelity(), "max_bond": max(m.bond_dims())}
    m.close()
    return out


def xy_run(lib, dims, chi, prec, grow=1):
    """The XY workload: open Lx x Ly grid, one qubit per site, g = 1, the initial state of Eq.
    xy_init at g tau = 0.06 pi (three Trotter steps of g dtau = 0.02 pi, then the staggered Z
    phases pi/8), quench steps of g dt = 0.05 pi (every gate by SWAP routing); `grow` untimed
    steps, then one step timed with CUDA events on the handle's stream."""
    import torch
    Lx, Ly = (int(v) for v in dims.split("x"))
    g, dt, dtau = 1.0, 0.05 * math.pi, 0.02 * math.pi
    s = torch.cuda.Stream()
    m = lib.MPS(lib.xy_config(Lx, Ly, chi, g, dt, prec=prec), stream=s.cuda_stream)
    m.step(g, 0.0, dtau, 2, 3)
    m.apply_layer(lib.LAYER_ZSTAG, math.pi / 8)
    m.step(g, 0.0, dt, 2, grow)
    u0 = m.stats()["truncations"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    m.step(g, 0.0, dt, 2, 1)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    u = m.stats()["truncations"] - u0
    out = {"workload": "XY model %dx%d open grid, one qubit per site, chi=%d, g tau=0.06 pi, g dt=0.05 pi, SWAP "
                       "routing, %d untimed quench step(s) then one timed" % (Lx, Ly, chi, grow),
           "precision": prec, "two_site_updates_per_s": u / (ms / 1e3), "ms_per_step": ms,
           "two_site_updates_per_step": u, "F": m.fidelity(), "X_stag2": m.expect(lib.X_STAG2),
           "max_bond": max(m.bond_dims())}
    m.close()
    return out


def cpu_baseline(Lx, Ly, chi, n_updates):
    smp = OracleSample(Lx, Ly, chi)
    phi = J * DT
    n = 0
    secs = 0.0
    for _ in range(max(1, n_updates)):
        k, t = smp.update(phi)
        n += k
        secs += t
    cores = len(os.sched_getaffinity(0))
    return {"value": n / secs, "unit": "bond updates/s", "cores": cores, "kind": "oracle",
            "sample": smp.describe(n, secs)}


def run_reference(args, Lx, Ly):
    """The oracle as the reference arm: each step is one bond update at the identical shape
    (OracleSample); W untimed steps, then K timed ones."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    smp = OracleSample(Lx, Ly, args.chi)
    phi = J * DT
    for _ in range(args.warmup):
        smp.update(phi)
    n = 0
    secs = 0.0
    for _ in range(args.steps):
        k, t = smp.update(phi)
        n += k
        secs += t
    value = n / secs
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": "bond updates/s at %dx%d chi=%d" % (Lx, Ly, args.chi), "value": value,
            "unit": "bond updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "TFIM %dx%d grouped MPS, bond updates at chi=%d (every bond at chi), one "
                                   "adjacent gate per step; J=-1 h=2 dt=0.25" % (Lx, Ly, args.chi)},
            "cpu_baseline": {"value": value, "unit": "bond updates/s", "cores": cores, "kind": "oracle",
                             "sample": smp.describe(n, secs)},
            "e2e": {"value": value, "unit": "bond updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fp64_form_rate(lib, m_split, Lx, Ly, n_updates, stream):
    """The FP64 form (complex128, exact SVD truncation) on the evolved state of the timed run:
    the split-form MPS is written to a checkpoint, converted to complex128 and loaded as an FP64
    handle, which then applies adjacent gates between the middle blocks; device time by CUDA
    events on its stream."""
    import torch

    gates = middle_adjacent_gates(lib.schedule_gates(Lx, Ly), Lx)
    with tempfile.TemporaryDirectory() as td:
        a = os.path.join(td, "split.bin")
        b = os.path.join(td, "fp64.bin")
        m_split.save(a)
        lib.convert_checkpoint(a, b, "fp64")
        g = lib.MPS.load_checkpoint(b, stream=stream.cuda_stream)
    phi = J * DT
    g.apply_gates(gates[0], 1, phi)  # brings the centre next to the middle blocks (untimed)
    torch.cuda.synchronize()
    st0 = g.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(n_updates):
        g.apply_gates(gates[(i + 1) % len(gates)], 1, phi)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n = g.stats()["truncations"] - st0["truncations"]
    g.close()
    return {"value": n / (ms / 1e3), "unit": "bond updates/s", "bond_updates": n, "ms": ms,
            "sample": "FP64 form (complex128 storage, FP64 GEMMs, exact truncation by one-sided Jacobi SVD) on the "
                      "evolved %dx%d state at chi=%d: %d adjacent gate(s) between the middle blocks" %
                      (Lx, Ly, m_split.cfg.chi_max, n)}


def one_gate(path, Lx, Ly):
    """One bond-update unit of the bench step on a saved state: the checkpoint is loaded on a
    stream of its own and the first adjacent gate between the middle blocks is applied once;
    device time by CUDA events, launches by the library's counter."""
    import torch
    from paper_2511_23438_gb300 import lib
    lib.load()
    s = torch.cuda.Stream()
    g = lib.MPS.load_checkpoint(path, stream=s.cuda_stream)
    gates = middle_adjacent_gates(lib.schedule_gates(Lx, Ly), Lx)
    torch.cuda.synchronize()
    l0, u0 = lib.launch_count(), g.stats()["truncations"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    g.apply_gates(gates[0], 1, J * DT)
    e1.record(s)
    torch.cuda.synchronize()
    out = {"one_gate_ms": e0.elapsed_time(e1), "launches": lib.launch_count() - l0,
           "bond_updates": g.stats()["truncations"] - u0, "launches_before": l0}
    g.close()
    return out


def other_split_rate(lib, m_split, prec, stream):
    """Another complex64 form on the evolved state of the timed run: the MPS is written to a
    checkpoint, relabelled with the form `prec` (same complex64 storage) and loaded on the same
    stream; one whole Trotter step is timed with CUDA events."""
    import torch

    with tempfile.TemporaryDirectory() as td:
        a = os.path.join(td, "a.bin")
        b = os.path.join(td, "b.bin")
        m_split.save(a)
        lib.convert_checkpoint(a, b, prec)
        g = lib.MPS.load_checkpoint(b, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    st0 = g.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(J, HX, DT, ORDER, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n = g.stats()["truncations"] - st0["truncations"]
    o = g.observables()
    g.close()
    return {"precision": prec, "value": n / (ms / 1e3), "unit": "bond updates/s", "bond_updates": n, "ms": ms,
            "sample": "one Trotter step of the evolved state of the timed run", "Z": o["Z"], "Z2": o["Z2"]}


def split_error_table(spec, prec, Lx=5, Ly=6, perturb=0.0):
    """Error of a complex64 form against the FP64 GPU form (both through the library, the FP64
    form being the one held to 1e-9 of the oracle) on the 5x6 grid (rows 3 + 3, d = 8) from the
    mid-temperature product state: for each chi, `steps` second-order steps side by side, the
    largest |d<Z_tot>|, |d<Z_tot^2>|, |d<X_tot>| and |dF/F| over the steps.  perturb != 0 starts
    the compared handle at theta + perturb (with prec fp64 this measures how far a perturbation
    of that size carries through the truncations of the run)."""
    from paper_2511_23438_gb300 import lib
    lib.load()
    theta = lib.initial_theta(J, HX, TEMP_DTHETA)
    rows = []
    for item in spec.split(","):
        chi, steps = (int(v) for v in item.split(":"))
        a = lib.MPS(lib.config(Lx, Ly, chi, theta, prec="fp64"))
        b = lib.MPS(lib.config(Lx, Ly, chi, theta + perturb, prec=prec))
        err = {"Z": 0.0, "Z2": 0.0, "X": 0.0, "F_rel": 0.0}
        t0 = time.perf_counter()
        for _ in range(steps):
            a.step(J, HX, DT, ORDER, 1)
            b.step(J, HX, DT, ORDER, 1)
            oa, ob = a.observables(), b.observables()
            for k in ("Z", "Z2", "X"):
                err[k] = max(err[k], abs(oa[k] - ob[k]))
            err["F_rel"] = max(err["F_rel"], abs(b.fidelity() / a.fidelity() - 1))
        rows.append({"chi": chi, "steps": steps, "F_fp64": a.fidelity(), "max_bond": max(a.bond_dims()),
                     "max_abs_err": err, "s": time.perf_counter() - t0})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        a.close()
        b.close()
    return {"split_error": rows, "precision": prec, "perturb": perturb, "grid": "%dx%d" % (Lx, Ly),
            "reference": "FP64 GPU form (complex128, exact SVD truncation)"}


def reduce_over_ranks(ms, updates, dist, device):
    """Replicas: the job's time is the slowest rank's timed region, its work the sum of all
    ranks' bond updates (no collective touches the data path; this is the only one)."""
    import torch

    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    u = torch.tensor([float(updates)], device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.item(), u.item()


def main():
    args = parse()
    Lx, Ly = (int(x) for x in args.grid.split("x"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, Lx, Ly)
        return
    if args.peaks:
        print(json.dumps(measure_peaks()), flush=True)
        return
    if args.one_gate:
        print(json.dumps(one_gate(args.one_gate, Lx, Ly)), flush=True)
        return
    if args.split_error:
        print(json.dumps(split_error_table(args.split_error, args.prec, perturb=args.split_perturb)), flush=True)
        return

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2511_23438_gb300 import build, lib

    build.build()
    lib.load()
    stream = torch.cuda.Stream()
    theta = lib.initial_theta(J, HX, TEMP_DTHETA)
    cfg = lib.config(Lx, Ly, args.chi, theta, prec=args.prec, J=J, h=HX, dt=DT, order=ORDER, seed=20261203 + rank)
    m = lib.MPS(cfg, stream=stream.cuda_stream)
    for _ in range(args.warmup):
        m.step(J, HX, DT, ORDER, 1)
        m.observables()
    torch.cuda.synchronize()

    # ---- device-timed region: K steps, inputs resident in HBM
    clocks = ClockSampler(local)
    clocks.start()
    st0 = m.stats()
    cnt0 = m.counters()
    l0 = lib.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    obs = None
    for _ in range(args.steps):
        m.step(J, HX, DT, ORDER, 1)
        obs = m.observables()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = lib.launch_count() - l0
    st1 = m.stats()
    cnt1 = m.counters()
    clk = clocks.stop()
    # one more step with per-launch-site CUDA-event timing (kept out of the timed region)
    lib.kernel_timing(True)
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    m.step(J, HX, DT, ORDER, 1)
    m.observables()
    ev3.record(stream)
    torch.cuda.synchronize()
    ktimes = lib.kernel_times()
    lib.kernel_timing(False)
    kstep_ms = ev2.elapsed_time(ev3)
    updates = st1["truncations"] - st0["truncations"]
    ms_max, upd_all = reduce_over_ranks(ms, updates, dist, "cuda")
    value = upd_all / (ms_max / 1e3)

    # ---- end to end through the C ABI: per step the layer parameters go host -> device (the
    # in-block unitaries the library uploads) and the observables + F come back to the host
    e2e_steps = max(1, args.steps // 2)
    st0 = m.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        m.step(J, HX, DT, ORDER, 1)
        m.observables()
        m.fidelity()
    e2e_s = time.perf_counter() - t0
    e2e_updates = m.stats()["truncations"] - st0["truncations"]
    nblk = 2 * Lx
    elem = 16 if args.prec == "fp64" else 8
    h2d = 2 * nblk * 1024 * elem  # two local layers per step, one 32x32 slot per block
    d2h = 4 * 8 + e2e_updates // max(1, e2e_steps) * 2 * 2 * args.chi * (8 if args.prec == "fp64" else 4)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # ---- roofline of the dominant launch site (device time from CUDA events on the handle's stream)
    peaks = read_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6792.1)
    tc_peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1715.0))
    # FP32 CUDA-core peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz
    # (the measured FP32 matmul rate, bench.py --peaks, is 69.9); FP64: the measured matmul rate
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    fp64_peak = 1.10

    def roofline(name, kms, kn, kwork):
        if kms <= 0:
            return None
        if "in-block gate" in name:  # bytes
            r = {"bound": "hbm", "achieved": kwork / (kms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                 "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
        elif "tcgen05" in name:  # useful complex flops; the tensor pipe executes 3 bf16 products each
            r = {"bound": "tensor", "achieved": 3 * kwork / (kms / 1e3) / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
                 "useful_tflops": kwork / (kms / 1e3) / 1e12,
                 "peak_source": "measured (MEASURED_PEAKS.json bf16 sustained)"}
        else:  # CUDA-core arithmetic (the Householder reduction counted as 16 n^3 / 3 flops per launch)
            fp64 = args.prec == "fp64"
            pk = fp64_peak if fp64 else fp32_peak
            r = {"bound": "alu", "achieved": kwork / (kms / 1e3) / 1e12, "peak": pk, "unit": "TFLOP/s",
                 "peak_source": "measured FP64 matmul rate" if fp64 else
                 "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz"}
        r["frac"] = r["achieved"] / r["peak"]
        r["traffic"] = None
        if "hetrd" in name and args.prec != "fp64" and args.chi == 1024:
            # ncu DRAM bytes (read + write) of one n = 2048 complex64 launch, the core size of this
            # configuration (the matrix is read from HBM once)
            r["traffic"] = 34.56e6
            r["traffic_case"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum, one n = 2048 launch"
        r["kernel"] = name
        r["launches"] = kn
        r["avg_launch_ms"] = kms / max(1, kn)
        r["share_of_step"] = kms / kstep_ms
        return r

    dom = max(ktimes.items(), key=lambda kv: kv[1][0])
    roof = roofline(dom[0], *dom[1])
    tc = [(k, v) for k, v in ktimes.items() if "tcgen05" in k]
    roof_tc = roofline(tc[0][0], *tc[0][1]) if tc and tc[0][1][0] > 0 else None
    line = {"metric": "bond updates/s at %dx%d chi=%d" % (Lx, Ly, args.chi), "value": value,
            "unit": "bond updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "c128", "fp32": "c64", "split_bf16x3": "c64+bf16x3"}.get(args.prec, "c64"),
            "data": "synthetic",
            "config": {"workload": "TFIM %dx%d grouped MPS (d=%d, %d blocks), chi=%d, mid temperature "
                                   "(dtheta=2pi/9), J=-1 h=2 dt=0.25, 2nd-order Trotter, precision %s"
                                   % (Lx, Ly, 2 ** ((Ly + 1) // 2), 2 * Lx, args.chi, args.prec),
                       "l2": "inputs larger than L2 (MPS resident in HBM, streamed every step)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "gpu_launches": launches,
            "launches_before_timed": l0,
            "bond_updates": int(upd_all),
            "observables": obs,
            "clocks": clk,
            "roofline": roof,
            "roofline_tensorcore_gemm": roof_tc,
            "e2e": {"value": e2e_updates / e2e_s, "unit": "bond updates/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "kernel_sites_ms": {k: round(v[0], 3) for k, v in ktimes.items()},
            "kernel_sites_tflops": {k: round(v[2] / (v[0] / 1e3) / 1e12, 3) for k, v in ktimes.items()
                                    if v[0] > 0 and v[2] > 0 and "in-block" not in k},
            "counters_per_step": {k: (cnt1[k] - cnt0[k]) / args.steps for k in cnt1}}
    if args.save_state and world == 1:
        m.save(args.save_state)
    if args.fp64_updates > 0 and world == 1:
        line["fp64_form"] = fp64_form_rate(lib, m, Lx, Ly, args.fp64_updates, stream)
    if args.other_split and world == 1 and args.prec != args.other_split:
        line["other_split_form"] = other_split_rate(lib, m, args.other_split, stream)
    m.close()
    if args.serve_jobs > 0 and world == 1:
        line["serve"] = serve_run(args.serve_jobs, args.serve_steps, args.prec)
    if args.batch_mps > 0 and world == 1:
        line["batched"] = batched_run(lib, args.batch_mps, args.prec)
    if args.three_d and world == 1:
        line["three_d"] = three_d_run(lib, args.three_d, args.three_d_chi, args.prec)
    if args.xy and world == 1:
        line["xy"] = xy_run(lib, args.xy, args.xy_chi, args.prec)
    if not args.no_cpu_baseline and world == 1:  # the oracle baseline is timed at N = 1 only
        line["cpu_baseline"] = cpu_baseline(Lx, Ly, args.chi, args.cpu_updates)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
