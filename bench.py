#!/usr/bin/env python3
"""Benchmark: CG iterations/s of the adhesive 2048 x 2048 load-unload sweep.

Workload (one "step"): graded half-space k = 0.3, nu = 0.3, E0 = c0 = 1, domain
side 1 on 2048 x 2048 square elements; rigid paraboloid R = 1 centred;
non-adhesive preload to d0 = +0.02, then 400 adhesive pull-off steps of
1.1e-4 (to d = -0.024, past pull-off) with work of adhesion 1e-3 (Sec. 3.1
algorithm, Eq. 24 with Table 1's c1).  Precision FP32 + FP64 refinement (the
mode whose pressures meet 1e-5 relative L2 against FP64 on every workload):
FP32 transform passes and fields, FP64 scalars, and every detach round's
pressure refined against the FP64 residual before the detach decision.
Inputs are synthetic (the paraboloid), resident in HBM for `value`.

value       : CG iterations of all ranks / max-over-ranks device time (CUDA
              events); every fixed-set CG iteration counts, those of the
              refinement's correction solves included
e2e         : the same through the C ABI with pinned host buffers (profile in,
              per-step results and the final pressure out), wall clock
roofline    : the dominant transform pass, algorithmic bytes / its live average
              duration (CUDA events recorded inside the captured CG graphs); the
              library counts each timed launch's bytes and flops from the torus
              and rows that launch worked on (bem_pass_work).  `traffic` is the
              ncu DRAM bytes per launch of that kernel from profiles/, or null
              when the kernel sources changed since that capture
plain_fp32  : the same sweep in plain FP32 (no refinement), and how its
              contact counts and forces compare with the timed sweep's
full_torus  : the 2048^2 Polonsky-Keer step as the paper applies it, on the whole
              4096^2 torus: a non-adhesive rough-surface solve whose overlap set
              spans the grid; CG iterations/s and HBM GB/s at 128 N^2 bytes per
              iteration (two transforms plus the CG fields), and the FP32 and
              FP32 + refinement pressures against the FP64 solve's
cpu_baseline: the FP64 oracle on a bounded sample of the same unit of work
              (fixed-set CG iterations of an unloading step on the full 2048^2
              grid, one 4096^2 FFT transform each), on all host cores

batch       : (rank 0, one GPU) the seeded mix of 256 independent solves
              through the native request server at FP32 + FP64 refinement,
              against the plain FP64 path one solve at a time
serving     : the Poisson request stream (200/s) through the server, and the
              plain FP64 path on its first requests: solves/s, p50/p99 latency
rough_4096  : (rank 0) the 4096^2 non-adhesive rough-surface solve on the 8192^2
              torus in each precision

--impl reference times the oracle alone (rank 0) on the same unit of work and
prints its own line.
"""
from __future__ import annotations

import argparse
import ctypes
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
# the unit of work both arms count: one fixed-set CG iteration of the sweep
UNIT_OF_WORK = "fixed-set CG iteration of the sweep's held-set solves (one 2048^2 FFT convolution each)"
L2_NOTE = "flushed between steps (256 MiB device write); the host arm has no device cache"
ORACLE_ITERS = 3  # oracle fixed-set CG iterations per reference step


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


def shared_config(world):
    """The `config` both arms print (same workload, grid and unit of work)."""
    return {"workload": WORKLOAD, "grid": [N, N], "unit_of_work": UNIT_OF_WORK,
            "parallelism": f"replicas x{world}", "l2": L2_NOTE}


def oracle_sample_desc(cores):
    return (f"{ORACLE_ITERS} fixed-set CG iterations (Sec. 3.1 held-set solve) per step at the first "
            "unloading depth of the 2048^2 sweep, on the full 4096^2 torus (oracle FFT mode, FP64, "
            f"scipy.fft on {cores} threads); held set = the preload's contact disc of the closed-form "
            "radius (Eq. 15), start p = 0; the initial residual transform is timed apart and excluded")


def run_reference(args, rank, world):
    """The oracle, as it stands, on the same unit of work as the GPU arm."""
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    per = []
    for s in range(args.warmup + args.steps):
        it, el = oracle_fixed_set_sample(ORACLE_ITERS, cores)
        if s >= args.warmup:
            per.append((it, el))
    its = sum(i for i, _ in per)
    tot = sum(e for _, e in per)
    v = its / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "precision": "fp64 (oracle)", "config": shared_config(world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": oracle_sample_desc(cores), "host": host_cpu()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


_ORACLE_CACHE = {}


def oracle_fixed_set_sample(iters, workers):
    """(iterations, seconds) of the oracle's fixed-set CG (Sec. 3.1) on the full
    2048^2 grid at the first unloading depth; the set-up residual transform is
    timed separately and subtracted."""
    import oracle
    from paper_1612_08395_gb300 import inputs
    key = ("conv", workers)
    if key not in _ORACLE_CACHE:
        dx = 1.0 / N
        Kq = oracle.influence_quarter(K_EXP, dx, dx, N + 1, N + 1)
        _ORACLE_CACHE[key] = oracle.FFTConvolver(Kq, N, N, workers=workers)
    conv = _ORACLE_CACHE[key]
    A = oracle.compliance(K_EXP, NU, E0, C0)
    h = inputs.paraboloid(N, R)
    a0 = oracle.closed_forms.hertz_radius(D0, K_EXP, R)
    S = inputs.radius_grid(N, N, 1.0 / N) <= a0
    c = h - (D0 - DD)
    p0 = np.zeros_like(h)
    t0 = time.perf_counter()
    oracle.fixed_set_cg(A, conv, c, S, p0, tol=0.0, max_iter=0)
    t1 = time.perf_counter()
    res = oracle.fixed_set_cg(A, conv, c, S, p0, tol=0.0, max_iter=iters)
    t2 = time.perf_counter()
    return res.iterations, max((t2 - t1) - (t1 - t0), 1e-9)


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
    # latency of each request, in request order
    lat = [c["t_end"] - c["t_submit"] + sub_late[c["tag"]][0]
           for c in sorted(comps, key=lambda c: sub_late[c["tag"]][1])]
    bad = [c["status"] for c in comps if c["status"] != 0]
    iters = sum(sum(r.iterations for r in c["results"]) for c in comps)
    return el, lat, iters, bad


def batch_and_serving(bem, inputs, n_batch, n_serve, n_serve_plain, workers):
    """Many independent solves: the seeded batch mix (grid sides 128..1024) and a
    Poisson request stream (rate 200/s, sides 64..2048), each through the server
    at FP32 + FP64 refinement and through the plain FP64 path one at a time (the
    stream's plain path on its first n_serve_plain requests)."""
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
            "workload": f"{n_batch} of the 256 seeded solves: side uniform in {{128,256,512,1024}}, "
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
        m = min(n_serve_plain, n_serve)
        el64, lat64, _ = _plain_fp64(bem, reqs[:m], a32[:m], arrivals=arr[:m])
        out["serving"] = {
            "workload": f"{n_serve} requests, Poisson arrivals at 200/s (seed 5), side "
                        "round(exp(U[ln 64, ln 2048])), k~U[-0.8,0.8], half adhesive; HBM budget 150 GB",
            "requests": n_serve, "solves_per_s": n_serve / el, "p50_ms": 1e3 * _pct(lat, 50),
            "p99_ms": 1e3 * _pct(lat, 99), "max_ms": 1e3 * max(lat), "precision": "fp32_refine",
            "workers": workers, "failed": bad, "latency": "completion minus arrival",
            "first_requests": {"n": m, "p50_ms": 1e3 * _pct(lat[:m], 50), "p99_ms": 1e3 * _pct(lat[:m], 99)},
            "plain_fp64": {"requests": m, "solves_per_s": m / el64, "p50_ms": 1e3 * _pct(lat64, 50),
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


def kernel_sources_sha():
    """sha256 of the transform kernels' sources (a traffic figure from profiles/
    is used only while they are unchanged)."""
    import hashlib
    hs = hashlib.sha256()
    for f in ("conv_kernels.cuh", "common.cuh", "geo_table.h", "bem_impl.h"):
        with open(os.path.join(ROOT, "paper_1612_08395_gb300", "csrc", f), "rb") as fh:
            hs.update(fh.read())
    return hs.hexdigest()[:16]


def profiled_traffic(kernel_key, bytes_per_launch):
    """ncu DRAM bytes per launch recorded in profiles/traffic_*.md for this kernel
    (lines `kernel_key:`, `source_sha16:`, `dram_bytes_per_launch:` and, when the
    captured launch worked on another number of rows than the average timed one,
    `algorithmic_bytes_of_that_launch:`), scaled to this run's average launch by
    algorithmic bytes; None if absent or taken on other kernel sources."""
    import glob
    sha = kernel_sources_sha()
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "traffic_*.md"))):
        kv = {}
        with open(f) as fh:
            for line in fh:
                if ":" in line and not line.startswith(("#", "|", " ")):
                    k, v = line.split(":", 1)
                    kv[k.strip().lstrip("- ").strip("`")] = v.strip().strip("`")
        if kv.get("kernel_key") == kernel_key and kv.get("source_sha16") == sha:
            try:
                dram = float(kv["dram_bytes_per_launch"])
                algo = float(kv.get("algorithmic_bytes_of_that_launch", "nan"))
            except (KeyError, ValueError):
                return None, None
            if algo > 0 and bytes_per_launch > 0:
                return dram * bytes_per_launch / algo, os.path.basename(f) + " (scaled by algorithmic bytes)"
            return dram, os.path.basename(f)
    return None, None


def full_torus_leg(bem, inputs, torch, hd, stream, hbm):
    """The 2048^2 Polonsky-Keer step on the whole 4096^2 torus: a non-adhesive
    rough-surface solve (config 3b's recipe at 2048^2, d = rms height) whose
    overlap set spans the grid, in FP32, FP32 + refinement and FP64."""
    rough_h, rough_d = inputs.rough_self_affine(N, hurst=0.8, q1_over_q0=256.0, rms_slope=0.1, seed=1612)
    rough_dev = torch.from_numpy(rough_h).cuda()
    out = {"workload": "non-adhesive self-affine rough surface (H=0.8, q1/q0=256, rms slope 0.1, seed 1612) "
                       "at d = rms height, 2048^2 grid, 4096^2 torus",
           "bytes_per_iteration": 128.0 * N * N,
           "bytes_model": "128 N^2: two transforms (44 N^2 each) and the CG fields (40 N^2), FP32"}
    ps = {}
    for prec in ("fp32", "fp32_refine", "fp64"):
        p = torch.empty((N, N), dtype=torch.float64, device="cuda")
        hd.solve(rough_dev, rough_d, pressure_out=p, precision=prec, stream=stream)  # warm-up
        torch.cuda.synchronize()
        hd.pass_times(reset=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, rc = hd.solve(rough_dev, rough_d, pressure_out=p, precision=prec, stream=stream,
                           time_passes=prec == "fp32")
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        ent = {"iterations": res.iterations, "ms": ms, "iter_per_s": 1e3 * res.iterations / ms,
               "contact_fraction": res.contact_count / (N * N), "force": res.force, "status": rc}
        if prec == "fp32":
            ent["hbm_gbs"] = ent["iter_per_s"] * out["bytes_per_iteration"] / 1e9
            ent["hbm_frac"] = ent["hbm_gbs"] / hbm
            wb, _ = hd.pass_work()
            pms, pn, _ = hd.pass_times(reset=True)
            if pn:
                avg = [m / pn for m in pms]
                ent["pass_us"] = {k: 1e3 * v for k, v in zip("ABC", avg)}
                ent["pass_gbs"] = {k: b / (v * 1e-3) / 1e9 for k, b, v in zip("ABC", wb, avg)}
                ent["pass_hbm_frac"] = {k: g / hbm for k, g in ent["pass_gbs"].items()}
        ps[prec] = p.cpu().numpy()
        out[prec] = ent
    ref = ps["fp64"]
    for prec in ("fp32", "fp32_refine"):
        out[prec]["pressure_rel_l2_vs_fp64"] = float(np.linalg.norm(ps[prec] - ref) / np.linalg.norm(ref))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32_refine", choices=["fp32", "fp32_refine", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-steps", type=int, default=NSTEPS,
                    help="unloading steps per sweep (400 = the workload; fewer only for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2, help="sweeps timed through the C ABI with host buffers")
    ap.add_argument("--batch-jobs", type=int, default=256,
                    help="solves of the batch mix to time (256 = the whole mix; 0 = skip)")
    ap.add_argument("--serve-requests", type=int, default=128,
                    help="requests of the Poisson stream to serve (0 = skip)")
    ap.add_argument("--serve-plain", type=int, default=32,
                    help="of those, how many the plain FP64 path serves for comparison")
    ap.add_argument("--workers", type=int, default=8, help="server worker streams")
    ap.add_argument("--no-rough-4096", action="store_true",
                    help="skip the 4096^2 rough-surface solves reported after the timed region")
    ap.add_argument("--no-side-legs", action="store_true",
                    help="skip plain_fp32 and full_torus (profiling runs only)")
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

    def one_sweep(precision, timed_passes=False, prof=prof_d, out=p_d, use_stream=True):
        res, rc = h.sweep(prof, ds, dgamma=DGAMMA, final_pressure=out, time_passes=timed_passes,
                          precision=precision, stream=stream if use_stream else None)
        return res

    for _ in range(args.warmup):
        one_sweep(args.precision)
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
        results = one_sweep(args.precision, timed_passes=True)
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
    e2e_steps = 0 if args.no_e2e else max(1, min(args.e2e_steps, args.steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(e2e_steps):
        res = one_sweep(args.precision, prof=prof_pin, out=out_pin, use_stream=False)
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
    kernel_key = f"pass {names[dom]}, fixed-set loop, FP32, box torus of the 2048^2 sweep"
    traffic, traffic_src = profiled_traffic(kernel_key, bytes_dom)

    forces = [r.force for r in results]
    counts = [r.contact_count for r in results]
    last_contact = max((i for i, c in enumerate(counts) if c > 0), default=0)
    sweep = {"precision": args.precision, "torus": [info.Px, info.Py],
             "fp32_shapes": {"rows_per_cta": info.rows_per_cta, "cols_per_cta": info.cols_per_cta,
                             "col_radix": info.col_radix},
             "sweep_s": elapsed / args.steps, "cg_iterations_per_step": iters_total / args.steps,
             "detach_rounds": int(sum(r.detach_rounds for r in results)),
             "stalled_solves": int(sum(r.stalled for r in results)),
             "pull_off_force": min(forces), "last_contact_depth": float(ds[last_contact]),
             "preload_force": forces[0], "preload_contact_count": counts[0]}

    side = {}
    if rank == 0 and not args.no_side_legs:
        # plain FP32 sweep: speed, and agreement with the timed (refined) sweep
        p32 = torch.empty_like(p_d)
        one_sweep("fp32", out=p32)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r32 = one_sweep("fp32", out=p32)
        e1.record(stream)
        e1.synchronize()
        ms32 = e0.elapsed_time(e1)
        it32 = sum(r.iterations for r in r32)
        fmax = max(abs(f) for f in forces)
        side["plain_fp32"] = {
            "sweep_s": ms32 / 1e3, "cg_iterations": it32, "iter_per_s": 1e3 * it32 / ms32,
            "steps_with_other_contact_count": int(sum(a.contact_count != b.contact_count
                                                      for a, b in zip(r32, results))),
            "max_force_diff_over_max_force": max(abs(a.force - b.force) for a, b in zip(r32, results)) / fmax,
            "compared_with": args.precision}
        side["full_torus"] = full_torus_leg(bem, inputs, torch, h, stream, hbm)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "fp32_refine" else ("f32" if args.precision == "fp32" else "f64"),
        "data": "synthetic", "precision": args.precision,
        "config": shared_config(world),
        "sweep": sweep,
        "roofline": {"kernel": f"pass {names[dom]}", "bound": "hbm", "achieved": achieved,
                     "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                     "traffic_source": traffic_src, "kernel_key": kernel_key,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                     "avg_ms": {k: v for k, v in zip(names, avg_ms)}, "timed_launches": pass_n,
                     "bytes_per_launch": bytes_dom,
                     "fixed_set_fraction": frac_cg,
                     "alu": {"achieved": flops_dom / (avg_ms[dom] * 1e-3) / 1e12,
                             "peak": fp32_peak_tflops(clocks.get("sm_max_mhz")), "unit": "TFLOP/s",
                             "frac": flops_dom / (avg_ms[dom] * 1e-3) / 1e12
                             / fp32_peak_tflops(clocks.get("sm_max_mhz")),
                             "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}},
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": UNIT, "steps": e2e_steps,
                "h2d_bytes_per_step": 8 * N * N + 8 * len(ds),
                "d2h_bytes_per_step": 8 * N * N + ctypes.sizeof(bem.Result) * len(ds)},
        "gpu_launches": int(launches),
    }
    line.update(side)
    if args.sweep_steps != NSTEPS:
        line["note"] = f"profiling run: {args.sweep_steps} unloading steps, not the workload"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        its, el = 0, 0.0
        for _ in range(2):
            i1, e1_ = oracle_fixed_set_sample(ORACLE_ITERS, cores)
            its += i1
            el += e1_
        line["cpu_baseline"] = {"value": its / el, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "2 x " + oracle_sample_desc(cores), "host": host_cpu()}
    h.close()
    del l2_flush
    if rank == 0 and world == 1 and not args.no_rough_4096:
        line.update(rough_4096(bem, inputs, torch))
    if rank == 0 and world == 1 and (args.batch_jobs or args.serve_requests):
        line.update(batch_and_serving(bem, inputs, args.batch_jobs, args.serve_requests, args.serve_plain,
                                      args.workers))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
