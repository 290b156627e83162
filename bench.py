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
bounded sample of the same workload and prints the same JSON line.
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
    ap.add_argument("--cpu-sample-chi", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=16, help="jobs of the short serving run (0: none)")
    ap.add_argument("--peaks", action="store_true", help="measure dense matmul rates (torch) and exit")
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


def serve_run(njobs, prec):
    """A short serving run: Poisson arrivals (20 jobs/s, seeded) over the grids of the serving
    mix, chi in {32, 64}, 4 second-order steps each, 8 slots, 8 GB budget."""
    from paper_2511_23438_gb300 import inputs, serve

    jobs = inputs.serving_jobs(njobs, rate=20.0, seed=20261203, chis=(32, 64), steps=4, prec=prec)
    res, st = serve.Server(serve.GpuEngine(), 8 << 30, max_slots=8).run(jobs)
    st["workload"] = ("%d jobs, Poisson 20/s, grids %s, chi {32,64}, 4 steps, %s, 8 slots, 8 GB budget"
                      % (njobs, "/".join("%dx%d" % g for g in inputs.SERVE_GRIDS), prec))
    return st


def cpu_baseline(Lx, Ly, sample_chi, dtheta):
    """The oracle, as it stands, on a bounded sample of the workload: the same grid at a reduced
    chi; one untimed Trotter step saturates the bonds, the second step (all of its bond updates
    and the observables) is timed.  The per-update cost grows ~chi^3."""
    from oracle import layout, model, mps

    th = model.initial_theta(dtheta)
    alpha, phi = model.layer_angles(J, HX, DT, ORDER)
    intra, inter = layout.schedule(Lx, Ly)
    m = mps.MPS(Lx, Ly, sample_chi, th)

    def step():
        m.x_layer(alpha)
        m.zz_intra(phi, intra)
        for g in inter:
            m.zz_inter(g, phi)
        m.x_layer(alpha)
        m.observables()

    step()
    n0 = len(m.fidelities)
    t0 = time.perf_counter()
    step()
    dt = time.perf_counter() - t0
    n_upd = len(m.fidelities) - n0
    cores = len(os.sched_getaffinity(0))
    return {"value": n_upd / dt, "unit": "bond updates/s", "cores": cores, "kind": "oracle",
            "sample": "oracle (NumPy FP64, LAPACK SVD): second Trotter step of %dx%d at chi=%d, bonds saturated "
                      "(%d bond updates + observables in %.1f s; same grid, reduced chi)"
                      % (Lx, Ly, sample_chi, n_upd, dt)}


def run_reference(args, Lx, Ly):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = []
    for _ in range(args.warmup + args.steps):
        steps.append(cpu_baseline(Lx, Ly, args.cpu_sample_chi, TEMP_DTHETA))
    timed = steps[args.warmup:]
    value = statistics.mean(s["value"] for s in timed)
    line = {"impl": "reference", "metric": "bond updates/s at %dx%d chi=%d" % (Lx, Ly, args.chi), "value": value,
            "unit": "bond updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "TFIM %dx%d grouped MPS, chi=%d (reference sampled at chi=%d), mid temperature, "
                                   "J=-1 h=2 dt=0.25, 2nd-order Trotter" % (Lx, Ly, args.chi, args.cpu_sample_chi)},
            "cpu_baseline": timed[-1],
            "e2e": {"value": value, "unit": "bond updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    fp32_peak = 69.9   # measured FP32 CUDA-core matmul rate of this GPU (bench.py --peaks)
    fp64_peak = 1.10   # measured FP64 matmul rate of this GPU (bench.py --peaks)

    def roofline(name, kms, kn, kwork):
        if kms <= 0:
            return None
        if "in-block gate" in name or "Householder" in name:  # bytes
            r = {"bound": "hbm", "achieved": kwork / (kms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                 "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
        elif "tcgen05" in name:  # useful complex flops; the tensor pipe executes 3 bf16 products each
            r = {"bound": "tensor", "achieved": 3 * kwork / (kms / 1e3) / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
                 "useful_tflops": kwork / (kms / 1e3) / 1e12,
                 "peak_source": "measured (MEASURED_PEAKS.json bf16 sustained)"}
        else:  # CUDA-core arithmetic
            pk = fp64_peak if args.prec == "fp64" else fp32_peak
            r = {"bound": "alu", "achieved": kwork / (kms / 1e3) / 1e12, "peak": pk, "unit": "TFLOP/s",
                 "peak_source": "measured (torch matmul, bench.py --peaks)"}
        r["frac"] = r["achieved"] / r["peak"]
        r["traffic"] = None
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
            "bond_updates": int(upd_all),
            "observables": obs,
            "clocks": clk,
            "roofline": roof,
            "roofline_tensorcore_gemm": roof_tc,
            "e2e": {"value": e2e_updates / e2e_s, "unit": "bond updates/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "kernel_sites_ms": {k: round(v[0], 3) for k, v in ktimes.items()}}
    if args.serve_jobs > 0 and world == 1:
        line["serve"] = serve_run(args.serve_jobs, args.prec)
    if not args.no_cpu_baseline and world == 1:  # the oracle baseline is timed at N = 1 only
        line["cpu_baseline"] = cpu_baseline(Lx, Ly, args.cpu_sample_chi, TEMP_DTHETA)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
