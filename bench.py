#!/usr/bin/env python3
"""Benchmark: CG iterations/s of the adhesive 2048 x 2048 load-unload sweep.

Workload (one "step"): graded half-space k = 0.3, nu = 0.3, E0 = c0 = 1, domain
side 1 on 2048 x 2048 square elements; rigid paraboloid R = 1 centred;
non-adhesive preload to d0 = +0.02, then 400 adhesive pull-off steps of
1.1e-4 (to d = -0.024, past pull-off) with work of adhesion 1e-3 (Sec. 3.1
algorithm, Eq. 24 with Table 1's c1).  FP32 transform passes, FP64 scalars.
Inputs are synthetic (the paraboloid), resident in HBM for `value`.

value       : CG iterations of all ranks / max-over-ranks device time (CUDA events)
e2e         : the same through the C ABI with pinned host buffers (profile in,
              pressure out), wall clock around the call
roofline    : the dominant transform pass, algorithmic bytes / its live average
              duration (CUDA events recorded inside the captured CG graphs); the
              library counts each timed launch's bytes and flops from the torus
              and rows that launch worked on (bem_pass_work)
roofline_full_torus : the same for the passes of a non-adhesive rough-surface
              solve on the same grid after the timed region, whose overlap set
              spans the grid: every launch transforms the whole 4096^2 torus
              (the sweep's solves run on the contact box's smaller torus)
cpu_baseline: the FP64 oracle (numpy FFT mode) on a bounded sample of the same
              workload, on this host's cores

batch       : (rank 0, one GPU) the seeded batch mix of independent solves
              through the native request server at FP32 + FP64 refinement,
              against the plain FP64 path one solve at a time; solves/s and
              the largest final-pressure difference between the two
serving     : the Poisson request stream (200/s) through the server and through
              the plain FP64 path: solves/s and p50/p99 latency from arrival
rough_4096  : (rank 0) the 4096^2 non-adhesive rough-surface solve on the 8192^2
              torus in each precision: CG iterations/s, contact fraction, force,
              and the passes' durations and bandwidth

--impl reference times the oracle alone (rank 0) and prints its own line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 2048
K_EXP, NU, E0, C0 = 0.3, 0.3, 1.0, 1.0
R = 1.0
DGAMMA = 1e-3
D0 = 0.02
DD = 1.1e-4
NSTEPS = 400
WORKLOAD = "adhesive paraboloid load-unload 2048x2048 (k=0.3, nu=0.3, R=1, dgamma=1e-3, d0=0.02, 400 steps of 1.1e-4)"
METRIC = "CG iterations/s, adhesive 2048^2 load-unload sweep"
UNIT = "iter/s"


def d_steps(nsteps=NSTEPS):
    return np.array([D0] + [D0 - DD * j for j in range(1, nsteps + 1)])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def fp32_peak_tflops(sm_mhz):
    """FP32 vector peak: 152 SMs x 128 lanes x 2 flops (FMA) x clock."""
    return 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


def aggregate(elapsed_s, iters, world, device):
    """Whole-job figures over ranks: (max elapsed seconds, total iterations).

    Every rank calls it after its timed region; with one rank it is the identity.
    """
    if world <= 1:
        return float(elapsed_s), float(iters)
    import torch
    import torch.distributed as dist
    el = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    it = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    dist.barrier()
    dist.all_reduce(el, op=dist.ReduceOp.MAX)
    dist.all_reduce(it, op=dist.ReduceOp.SUM)
    return float(el.item()), float(it.item())


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    per = []
    for s in range(args.warmup + args.steps):
        it, el, _ = cpu_oracle_sample_cached(2)
        if s >= args.warmup:
            per.append((it, el))
    its = sum(i for i, _ in per)
    tot = sum(e for _, e in per)
    v = its / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64 (oracle)",
                                            "grid": [N, N], "torus": [2 * N, 2 * N],
                                            "parallelism": "rank 0 only", "l2": "n/a (host)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "2 Polonsky-Keer CG iterations of the 2048^2 preload per step "
                                       "(oracle FFT mode, numpy pocketfft FP64, single thread)",
                             "host": host_cpu()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


_ORACLE_CACHE = {}


def cpu_oracle_sample_cached(iters):
    import oracle
    from paper_1612_08395_gb300 import inputs
    if "conv" not in _ORACLE_CACHE:
        dx = 1.0 / N
        Kq = oracle.influence_quarter(K_EXP, dx, dx, N + 1, N + 1)
        _ORACLE_CACHE["conv"] = oracle.FFTConvolver(Kq, N, N)
    conv = _ORACLE_CACHE["conv"]
    A = oracle.compliance(K_EXP, NU, E0, C0)
    h = inputs.paraboloid(N, R)
    t0 = time.perf_counter()
    res = oracle.pk_solve(A, conv, h, D0, tol=1e-300, max_iter=iters)
    return res.iterations, time.perf_counter() - t0, 0.0


def host_cpu():
    """nproc and the CPU model of this host, for the oracle's timing."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu": model}


def _pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if v else None


def _job_arrays(inputs, jobs):
    out = []
    for j in jobs:
        h, ds = inputs.job_profile(j)
        out.append((h, ds, np.empty((j["n"], j["n"]))))
    return out


def _plain_fp64(bem, jobs, arrays, arrivals=None):
    """One request at a time through a fresh FP64 handle (spectrum set-up included),
    in order; a request starts at its arrival time or when the previous one ends."""
    import torch
    lat, t0 = [], time.perf_counter()
    iters = 0
    for i, (j, (h, ds, p)) in enumerate(zip(jobs, arrays)):
        if arrivals is not None:
            while time.perf_counter() - t0 < arrivals[i]:
                time.sleep(1e-4)
        n = j["n"]
        with bem.Handle(n, n, 1.0 / n, 1.0 / n, j["k"], j["nu"]) as hd:
            res, rc = hd.sweep(h, ds, dgamma=j["dgamma"], final_pressure=p, precision="fp64")
        torch.cuda.synchronize()
        iters += sum(r.iterations for r in res)
        lat.append(time.perf_counter() - t0 - (arrivals[i] if arrivals is not None else 0.0))
    return time.perf_counter() - t0, lat, iters


def _served(bem, jobs, arrays, workers, budget, arrivals=None, precision="fp32_refine"):
    """All requests through the native server; with arrival times each is
    submitted when it arrives (Poisson stream), else all at once (a batch)."""
    comps, sub_late = [], {}
    with bem.Server(nworkers=workers, hbm_budget_bytes=budget) as srv:
        t0 = time.perf_counter()
        for i, (j, (h, ds, p)) in enumerate(zip(jobs, arrays)):
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[i]:
                    comps += srv.poll(wait_ms=0)
                    time.sleep(1e-4)
            n = j["n"]
            tag = srv.submit(n, n, 1.0 / n, 1.0 / n, j["k"], j["nu"], h, ds, dgamma=j["dgamma"],
                             final_pressure=p, precision=precision)
            sub_late[tag] = (time.perf_counter() - t0 - (arrivals[i] if arrivals is not None else 0.0), i)
        comps += srv.drain(1800.0)
        el = time.perf_counter() - t0
    lat = [c["t_end"] - c["t_submit"] + sub_late[c["tag"]][0] for c in comps]
    bad = [c["status"] for c in comps if c["status"] != 0]
    iters = sum(sum(r.iterations for r in c["results"]) for c in comps)
    return el, lat, iters, bad


def batch_and_serving(bem, inputs, n_batch, n_serve, workers):
    """Many independent solves: the seeded batch mix (grid sides 128..1024) and a
    Poisson request stream (rate 200/s, sides 64..2048), each through the server
    at FP32 + FP64 refinement and through the plain FP64 path one at a time."""
    budget = 150 << 30
    out = {}
    if n_batch:
        jobs = inputs.batch_jobs(256, seed=4)[:n_batch]
        a32 = _job_arrays(inputs, jobs)
        a64 = [(h, ds, np.empty_like(p)) for h, ds, p in a32]
        el, _, it32, bad = _served(bem, jobs, a32, workers, budget)
        el64, _, it64 = _plain_fp64(bem, jobs, a64)
        rel = [float(np.linalg.norm(x[2] - y[2]) / np.linalg.norm(y[2])) for x, y in zip(a32, a64)
               if np.linalg.norm(y[2]) > 0]
        out["batch"] = {
            "workload": f"first {n_batch} of 256 seeded solves: side uniform in {{128,256,512,1024}}, "
                        "k~U[-0.8,0.8], nu=0.3, paraboloid or rough, half adhesive (9-step unload)",
            "solves": n_batch, "solves_per_s": n_batch / el, "cg_iterations_per_s": it32 / el,
            "precision": "fp32_refine", "workers": workers, "failed": bad,
            "plain_fp64": {"solves_per_s": n_batch / el64, "cg_iterations_per_s": it64 / el64},
            "speedup_vs_plain_fp64": el64 / el,
            "final_pressure_rel_l2_vs_fp64_max": max(rel) if rel else None}
    if n_serve:
        reqs = inputs.serving_requests(n_serve, seed=5)
        arr = [r["arrival"] for r in reqs]
        a32 = _job_arrays(inputs, reqs)
        el, lat, it32, bad = _served(bem, reqs, a32, workers, budget, arrivals=arr)
        el64, lat64, _ = _plain_fp64(bem, reqs, a32, arrivals=arr)
        out["serving"] = {
            "workload": f"{n_serve} requests, Poisson arrivals at 200/s (seed 5), side "
                        "round(exp(U[ln 64, ln 2048])), k~U[-0.8,0.8], half adhesive; HBM budget 150 GB",
            "requests": n_serve, "solves_per_s": n_serve / el, "p50_ms": 1e3 * _pct(lat, 50),
            "p99_ms": 1e3 * _pct(lat, 99), "precision": "fp32_refine", "workers": workers,
            "failed": bad, "latency": "completion minus arrival",
            "plain_fp64": {"solves_per_s": n_serve / el64, "p50_ms": 1e3 * _pct(lat64, 50),
                           "p99_ms": 1e3 * _pct(lat64, 99)}}
    return out


def rough_4096(bem, inputs, torch, precisions=("fp32", "fp32_refine", "fp64")):
    """The 4096^2 non-adhesive workload: one solve of the seeded self-affine
    surface (H = 0.8, q1/q0 = 256, rms slope 0.1, PCG64 seed 1612) at d = rms
    height, k = 0.3, nu = 0.3, on the 8192^2 torus, per precision: CG iterations/s
    over the whole solve (CUDA events; the first solve of each precision is a
    warm-up), contact fraction and force, and the passes' average durations and
    bandwidth from the live pass timing."""
    n = 4096
    dx = 1.0 / n
    hgt, zrms = inputs.rough_self_affine(n, hurst=0.8, q1_over_q0=256.0, rms_slope=0.1, seed=1612)
    h_dev = torch.from_numpy(hgt).cuda()
    p_dev = torch.empty((n, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    hbm, _ = peaks()
    out = {"workload": "non-adhesive self-affine rough surface 4096x4096 (H=0.8, q1/q0=256, rms slope 0.1, "
                       "seed 1612), d = rms height, k=0.3, nu=0.3, 8192^2 torus"}
    with bem.Handle(n, n, dx, dx, K_EXP, NU, E0, C0) as hd:
        for prec in precisions:
            hd.solve(h_dev, zrms, pressure_out=p_dev, precision=prec, stream=stream)
            torch.cuda.synchronize()
            hd.pass_times(reset=True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res, rc = hd.solve(h_dev, zrms, pressure_out=p_dev, precision=prec, stream=stream,
                               time_passes=prec != "fp32_refine")
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            entry = {"iterations": res.iterations, "ms": ms, "iter_per_s": 1e3 * res.iterations / ms,
                     "contact_fraction": res.contact_count / (n * n), "force": res.force, "status": rc}
            if prec != "fp32_refine":
                wb, _ = hd.pass_work()
                pms, pn, _ = hd.pass_times(reset=True)
                if pn:
                    avg = [m / pn for m in pms]
                    entry["pass_us"] = {k: 1e3 * v for k, v in zip("ABC", avg)}
                    entry["pass_gbs"] = {k: b / (v * 1e-3) / 1e9 for k, b, v in zip("ABC", wb, avg)}
                    entry["pass_hbm_frac"] = {k: g / hbm for k, g in entry["pass_gbs"].items()}
            out[prec] = entry
    return {"rough_4096": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_refine", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-steps", type=int, default=NSTEPS,
                    help="unloading steps per sweep (400 = the workload; fewer only for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-jobs", type=int, default=64,
                    help="solves of the batch mix to time (256 = the whole mix; 0 = skip)")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests of the Poisson stream to serve (0 = skip)")
    ap.add_argument("--workers", type=int, default=8, help="server worker streams")
    ap.add_argument("--no-rough-4096", action="store_true",
                    help="skip the 4096^2 rough-surface solves reported after the timed region")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    from paper_1612_08395_gb300 import bem, build, inputs
    build.build()
    dx = 1.0 / N
    prof_h = inputs.paraboloid(N, R)
    prof_d = torch.from_numpy(prof_h).cuda()
    p_d = torch.empty((N, N), dtype=torch.float64, device="cuda")
    ds = d_steps(args.sweep_steps)
    stream = torch.cuda.current_stream()
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    h = bem.Handle(N, N, dx, dx, K_EXP, NU, E0, C0)
    info = h.info()
    opts = dict(precision=args.precision, stream=stream)

    def one_step(timed_passes=False):
        res, rc = h.sweep(prof_d, ds, dgamma=DGAMMA, final_pressure=p_d, time_passes=timed_passes,
                          **opts)
        return res

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # timed region
    sampler = ClockSampler(local)
    iters_total = 0
    launches0 = h.info().kernel_launches
    h.pass_times(reset=True)
    step_ms = []
    results = None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for _ in range(args.steps):
        l2_flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        results = one_step(timed_passes=True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        iters_total += sum(r.iterations for r in results)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = h.info().kernel_launches - launches0
    work_bytes, work_flops = h.pass_work()
    pass_ms, pass_n, pass_cg = h.pass_times(reset=True)
    elapsed = sum(step_ms) / 1e3
    elapsed_max, iters_all = aggregate(elapsed, iters_total, world, "cuda")
    value = iters_all / elapsed_max

    # e2e through the C ABI with pinned host buffers
    prof_pin = torch.from_numpy(prof_h).pin_memory()
    out_pin = torch.empty((N, N), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(0 if args.no_e2e else args.steps):
        res, rc = h.sweep(prof_pin, ds, dgamma=DGAMMA, final_pressure=out_pin,
                          precision=args.precision)
        e2e_iters += sum(r.iterations for r in res)
    e2e_s = time.perf_counter() - t0
    e2e_val = e2e_iters / e2e_s if e2e_iters else None

    # roofline of the dominant pass
    hbm, peak_src = peaks()
    avg_ms = [m / max(pass_n, 1) for m in pass_ms]
    dom = int(np.argmax(avg_ms))
    names = ["A", "B", "C"]
    frac_cg = pass_cg / max(pass_n, 1)
    bytes_dom = work_bytes[dom]
    flops_dom = work_flops[dom]
    achieved = bytes_dom / (avg_ms[dom] * 1e-3) / 1e9

    # the full 4096^2 torus: passes of a non-adhesive rough-surface solve (its
    # overlap set {h <= d} spans the grid, so every iteration transforms the
    # whole torus), timed the same way, outside the timed region
    rough_h, rough_d = inputs.rough_self_affine(N, hurst=0.8, q1_over_q0=256.0, rms_slope=0.1, seed=1612)
    rough_dev = torch.from_numpy(rough_h).cuda()
    h.pass_times(reset=True)
    for _ in range(2):
        h.solve(rough_dev, rough_d, precision=args.precision, stream=stream, time_passes=True)
    torch.cuda.synchronize()
    fb, _ = h.pass_work()
    fms, fn, _ = h.pass_times(reset=True)
    favg = [m / max(fn, 1) for m in fms]
    fdom = int(np.argmax(favg))
    full = {"kernel": f"pass {names[fdom]}", "bound": "hbm",
            "achieved": fb[fdom] / (favg[fdom] * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": fb[fdom] / (favg[fdom] * 1e-3) / 1e9 / hbm,
            "avg_ms": {k: v for k, v in zip(names, favg)}, "bytes_per_launch": fb[fdom],
            "timed_launches": fn,
            "workload": "non-adhesive self-affine rough surface (H=0.8, q1/q0=256, rms slope 0.1, "
                        "seed 1612) at d = rms height, 2048^2 grid, 4096^2 torus"}

    forces = [r.force for r in results]
    counts = [r.contact_count for r in results]
    last_contact = max((i for i, c in enumerate(counts) if c > 0), default=0)
    if args.sweep_steps != NSTEPS:
        line_note = f"profiling run: {args.sweep_steps} unloading steps, not the workload"
    else:
        line_note = None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": args.precision, "grid": [N, N],
                   "torus": [info.Px, info.Py], "parallelism": f"replicas x{world}",
                   "fp32_shapes": {"rows_per_cta": info.rows_per_cta, "cols_per_cta": info.cols_per_cta},
                   "l2": "flushed between steps (256 MiB write)",
                   "cg_iterations_per_step": iters_total / args.steps,
                   "pull_off_force": min(forces), "last_contact_depth": float(ds[last_contact]),
                   "preload_force": forces[0], "preload_contact_count": counts[0]},
        "roofline": {"kernel": f"pass {names[dom]}", "bound": "hbm", "achieved": achieved,
                     "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                     "avg_ms": {k: v for k, v in zip(names, avg_ms)}, "timed_launches": pass_n,
                     "bytes_per_launch": bytes_dom,
                     "fixed_set_fraction": frac_cg,
                     "alu": {"achieved": flops_dom / (avg_ms[dom] * 1e-3) / 1e12,
                             "peak": fp32_peak_tflops(clocks.get("sm_max_mhz")), "unit": "TFLOP/s",
                             "frac": flops_dom / (avg_ms[dom] * 1e-3) / 1e12
                             / fp32_peak_tflops(clocks.get("sm_max_mhz")),
                             "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}},
        "roofline_full_torus": full,
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 8 * N * N + 8 * len(ds),
                "d2h_bytes_per_step": 8 * N * N + 56 * len(ds)},
        "gpu_launches": int(launches),
    }
    if line_note:
        line["note"] = line_note
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        it, el, _ = cpu_oracle_sample_cached(3)
        line["cpu_baseline"] = {"value": it / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "3 Polonsky-Keer CG iterations of the 2048^2 preload solve "
                                          "(oracle FFT mode, numpy pocketfft FP64, single thread)",
                                "host": host_cpu()}
    h.close()
    del l2_flush
    if rank == 0 and world == 1 and not args.no_rough_4096:
        line.update(rough_4096(bem, inputs, torch))
    if rank == 0 and world == 1 and (args.batch_jobs or args.serve_requests):
        line.update(batch_and_serving(bem, inputs, args.batch_jobs, args.serve_requests, args.workers))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
