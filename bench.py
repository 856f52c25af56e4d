#!/usr/bin/env python3
"""Benchmark: DOF-steps/s of the implicit ADS/IGA Newmark step on one GB300.

Workload (one bench "step"): the 128^3-element scalar P-wave configuration,
p = 2 and p = 3 (one simulation each, 130^3 and 131^3 DOFs), tau = 2e-3,
200 Newmark steps per simulation, zero initial state, Ricker (f = 8,
t0 = 1/8) x Gaussian (sigma = 0.02) source at a seeded interior point, FP32
path (FP32 state and sweeps, FP64 1D factors).  DOF counts include boundary
coefficients.  The L2 cache is flushed (a 512 MB write) before every timed
step; inputs stay resident in HBM.

  value  : device time (CUDA events on the simulations' stream), whole job;
           both simulations advance together through ads_batch_step (one
           grouped launch per kernel and degree, the two degrees overlapping)
  e2e    : the same metric through the C ABI with pinned host buffers: per
           step set_state(u, v, a) of both simulations from host, 200 steps of
           both together (ads_batch_step), get_state of both to host
  fp64   : the FP64 path on the same workload (the path the FP32 one beats)
  roofline: dominant kernel, algorithmic bytes / its CUDA-event time
  cpu_baseline: the FP64 CPU oracle on a bounded sample of the workload
  elastic: the 96^3 elasticity configuration (p = 2, 100 steps), FP32 and FP64
  batch  : 64 uneven P-wave simulations (elements per axis U{32..160}, p in
           {2, 3}, tau in [1e-3, 5e-3], Gaussian pulses), 50 steps each, FP32,
           autotuned tiles, grouped launches replayed from CUDA graphs
  serving: 500 Poisson-arrival requests (20/s, 80% P-wave / 20% elasticity,
           grids log-uniform 24..256 per axis, 10..500 steps) under a 150 GB
           budget: p50/p99 latency and DOF-steps/s
  serving_saturated: the same requests at 2000/s under a 4 GB budget
           (admission waits on memory; the device is busy throughout)

--impl reference runs the CPU oracle as the reference arm (there is no
reference implementation of this paper; the oracle is the plain restatement).
Under torchrun (N > 1) every rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-steps/s (implicit ADS/IGA Newmark step, FP32 path)"
UNIT = "DOF-steps/s"
NE, NSTEPS, PS = 128, 200, (2, 3)
WORKLOAD = "pwave_ricker_128cubed_p2p3_200steps"

# algorithmic bytes per interior DOF of one launch (FP32): one read or write
# of each array element the kernel must touch
ALG_BYTES = {
    "rhs_xy_sweep": 8,      # read p, write x-and-y-swept field
    "rhs_x_sweep": 8,       # read p, write x-swept field
    "y_sweep": 8,           # read, write
    "z_sweep_update": 24,   # read swept field, p, q; write p, q, a (a is written in profiled steps)
}


def step_flops(p: int) -> dict:
    """Algorithmic FLOPs per interior unknown of one scalar-wave step (the
    method's own arithmetic, without the partitioned solve's corrections):
    RHS by sum factorisation 14(2p+1) + 3 (z: Mz, Kz; y: My, Ky, My; x: Kx,
    Mx; source and scale), each directional banded solve 4p + 1 (p FMAs
    forward, p back, one pivot multiply), the (p, q) update 3."""
    w = 2 * p + 1
    rhs, sweep, upd = 14 * w + 3, 4 * p + 1, 3
    return {"rhs": rhs, "sweep": sweep, "update": upd, "k1_fused": rhs + 2 * sweep,
            "step": rhs + 3 * sweep + upd}


def hbm_peak():
    """The measured HBM copy bandwidth of this machine's GPUs (GB/s) and its
    source, or the fallback figure."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measure_peaks(ads, local):
    """FMA throughput of the device's CUDA cores (ads_measure_fma_peak), with
    the clocks sampled while it runs."""
    out = {}
    with ClockSampler(local) as clk:
        for kind in ("ffma", "ffma2", "dfma"):
            vals = [ads.ads.measure_fma_peak(kind, local, 1 << 15 if kind == "dfma" else 1 << 17)[0]
                    for _ in range(3)]
            out[kind + "_tflops"] = round(max(vals), 2)
    out["clocks"] = clk.summary()
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 4 + i and r[4 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def max_over_ranks(x: float, ws: int) -> float:
    """The largest value of x over the ranks of the process group (the job
    takes as long as its slowest replica); x itself for one process."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, ws: int, t_max: float) -> float:
    """Whole-job throughput of ws independent replicas (weak scaling): all
    ranks' units over the slowest rank's time."""
    return units_per_rank * ws / t_max


def make_sims(precision, torch, ads, wl, stream=None):
    sims = []
    for p in PS:
        case = wl.ricker_case(ne=NE, p=p)
        sim = ads.Simulation(case.n_elem, case.p, case.tau, precision=precision, stream=stream)
        sim.set_source(case.source)
        sim.set_gaussian_state(None, None)
        sims.append(sim)
    return sims


def dofs(sim):
    return int(np.prod(sim.n))


def run_ours(args):
    import torch

    import paper_1911_08158_gb300 as ads
    from paper_1911_08158_gb300 import workloads as wl

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()   # all simulations and the timing events share it
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    sims = make_sims("fp32", torch, ads, wl, stream)
    # 0 trial steps: the first candidate (the fused single-CTA K1 when it
    # fits), a choice that does not depend on timings (for profiler runs)
    tiles = [s.autotune(args.autotune_steps) for s in sims]
    dof_steps = sum(dofs(s) for s in sims) * NSTEPS

    def bench_step():
        ads.batch_step(sims, NSTEPS)

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()

    # ---- timed region (device time per step, L2 flushed in between)
    times = []
    l0 = ads.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bench_step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        barrier()
        wall = time.perf_counter() - wall0
    launches = ads.launch_count() - l0
    t_dev = max_over_ranks(float(sum(times)), ws)
    value = replica_value(dof_steps * args.steps, ws, t_dev)

    # ---- per-kernel times (CUDA events between the kernels of single steps)
    kt = {}
    for s in sims:
        for _ in range(5):
            for name, ms in s.profile_step():
                kt.setdefault((name, s.p), []).append(ms)
    torch.cuda.synchronize()
    tot = {}
    for (name, p), v in kt.items():
        tot[name] = tot.get(name, 0.0) + float(np.mean(v))
    dom = max(tot, key=tot.get)
    # per launch of the dominant kernel, average over the two simulations:
    # K1 by back-to-back launches between one pair of events on the
    # simulations' stream (ads_profile_rhs; the events between the kernels of
    # a profiled step add a launch gap to every interval)
    per_launch, rhs_by_p = [], {}
    for s in sims:
        if dom == "rhs_xy_sweep":
            ms = float(np.median([s.profile_rhs(20) for _ in range(3)]))
            rhs_by_p["rhs_xy_sweep_p%d" % s.p] = round(ms, 5)
            m = [ms]
        else:
            m = [float(np.mean(v)) for (n, p), v in kt.items() if n == dom and p == s.p]
        if m:
            mx, my, mz = s.n[0] - 2, s.n[1] - 2, s.n[2] - 2
            per_launch.append((ALG_BYTES[dom] * mx * my * mz, m[0] / 1e3))
    alg_bytes = float(np.mean([b for b, _ in per_launch]))
    dur = float(np.mean([t for _, t in per_launch]))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg_bytes / dur / 1e9
    traffic = None   # ncu DRAM bytes per launch, from the committed summary of this kernel and workload
    try:
        import glob
        for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
            for line in open(path):
                f = line.split()
                if len(f) == 4 and f[0] == "traffic_bytes_per_launch" and f[1] == dom and f[2] == WORKLOAD:
                    traffic = int(f[3])
    except Exception:
        pass
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": "measured" if peaks else "fallback",
                "kernel_share": {k: round(v / sum(tot.values()), 4) for k, v in tot.items()},
                "kernel_ms": {k: round(v, 5) for k, v in tot.items()},
                "kernel_ms_by_p": {"%s_p%d" % (n, pp): round(float(np.mean(v)), 5) for (n, pp), v in kt.items()},
                "launch_ms_back_to_back": rhs_by_p}
    # the whole step: K1 reads p and writes x (8 B), K3 reads x, p, q and
    # writes p, q (20 B) per interior DOF; a is stored once per 16 steps
    interior = sum((s.n[0] - 2) * (s.n[1] - 2) * (s.n[2] - 2) for s in sims)
    step_gbs = interior * NSTEPS * args.steps * (28 + 4 / 16) / t_dev / 1e9
    roofline["step"] = {"bytes_per_interior_dof": 28.25, "achieved": round(step_gbs, 1),
                        "frac": round(step_gbs / peak, 4)}
    if dom == "rhs_xy_sweep" and rhs_by_p:
        # K1's arithmetic rate against the FP32 FMA peak (computed after the
        # peaks are measured, below)
        k1_fl = [step_flops(s.p)["k1_fused"] * (s.n[0] - 2) * (s.n[1] - 2) * (s.n[2] - 2) /
                 (rhs_by_p["rhs_xy_sweep_p%d" % s.p] / 1e3) / 1e12 for s in sims]
        roofline["k1_tflops_by_p"] = {"p%d" % s.p: round(v, 3) for s, v in zip(sims, k1_fl)}

    # ---- accuracy of both paths against the FP64 CPU oracle (fresh runs of
    # the whole configuration, 200 steps); the oracle runs in a thread during
    # the device-timed batch and elasticity measurements below
    acc = {}
    finals = {}
    s64 = make_sims("fp64", torch, ads, wl, stream)
    s32 = make_sims("fp32", torch, ads, wl, stream)
    for a, b in zip(s64, s32):
        a.step(NSTEPS)
        b.step(NSTEPS)
        ua = a.get_state(fields=("u",))[0]
        ub = b.get_state(fields=("u",))[0]
        finals[a.p] = (ua, ub)
        acc["p%d" % a.p] = float(np.linalg.norm(ub - ua) / np.linalg.norm(ua))

    # ---- FP64 path throughput (same workload, fewer steps; both simulations
    # advance together, as on the FP32 line)
    ads.batch_step(s64, 16)
    torch.cuda.synchronize()
    k64 = max(1, min(args.steps, 3))
    t64 = 0.0
    for _ in range(k64):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ads.batch_step(s64, NSTEPS)
        e1.record(stream)
        e1.synchronize()
        t64 += e0.elapsed_time(e1) / 1e3
    fp64 = {"value": dof_steps * k64 / t64, "ms_per_step": t64 / k64 * 1e3, "steps": k64}
    peaks_cc = measure_peaks(ads, local) if not args.no_peaks else {}
    # the FP64 path against the DFMA peak: algorithmic FLOPs of the step per
    # interior unknown times interior DOF-steps over the device time
    fl64 = sum(step_flops(s.p)["step"] * (s.n[0] - 2) * (s.n[1] - 2) * (s.n[2] - 2) for s in s64) * NSTEPS * k64
    if peaks_cc.get("dfma_tflops"):
        ach = fl64 / t64 / 1e12
        fp64["roofline"] = {"bound": "alu", "achieved": round(ach, 3), "peak": peaks_cc["dfma_tflops"],
                            "unit": "TFLOP/s", "frac": round(ach / peaks_cc["dfma_tflops"], 4),
                            "peak_source": "measured (ads_measure_fma_peak, DFMA)",
                            "flops_per_interior_dof_step": {"p%d" % p: step_flops(p)["step"] for p in PS}}

    # ---- end to end through the C ABI with pinned host buffers
    host = []
    for s in sims:
        bufs = [torch.zeros(s.shape, dtype=torch.float64).pin_memory() for _ in range(3)]
        u, v, a = s.get_state()
        for b, x in zip(bufs, (u, v, a)):
            b.copy_(torch.from_numpy(x))
        host.append(bufs)
    h2d = sum(3 * 8 * dofs(s) for s in sims)
    d2h = h2d
    lib = ads.library()
    ke = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        for s, bufs in zip(sims, host):
            ptr = [b.data_ptr() for b in bufs]
            ads.ads._check(lib.ads_set_state(s.handle, ptr[0], ptr[1], ptr[2], s.count, ads.ADS_HOST))
        ads.batch_step(sims, NSTEPS)   # both simulations together, as in the device-timed line
        for s, bufs in zip(sims, host):
            ptr = [b.data_ptr() for b in bufs]
            ads.ads._check(lib.ads_get_state(s.handle, ptr[0], ptr[1], ptr[2], s.count, ads.ADS_HOST))
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    e2e = {"value": dof_steps * ke * ws / te, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "steps": ke}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_elem": NE, "p": list(PS), "tau": 2e-3, "newmark_steps": NSTEPS,
                   "dofs": [dofs(s) for s in sims], "dof_steps_per_step": dof_steps, "k1_tile_rows": tiles,
                   "l2": "flushed (512 MB write) before each timed step", "parallelism": "replicas" if ws > 1 else "single"},
        "e2e": e2e, "gpu_launches": int(launches), "wall_s": wall,
        "fp64": fp64, "rel_l2_fp32_vs_fp64_u": acc,
        "roofline": roofline, "clocks": clk.summary(),
    }
    if peaks_cc:
        out["peaks_measured"] = peaks_cc
        if "k1_tflops_by_p" in roofline and peaks_cc.get("ffma2_tflops"):
            roofline["k1_frac_of_ffma2"] = {k: round(v / peaks_cc["ffma2_tflops"], 4)
                                            for k, v in roofline["k1_tflops_by_p"].items()}
    oracle_job = OracleFinals(PS, NSTEPS) if (rank == 0 and not args.no_oracle_check) else None
    if not args.no_batch:
        out["batch"] = guarded(run_batch, args, stream, flush)
    if not args.no_elastic:
        out["elastic"] = guarded(run_elastic, args, stream, flush)
    if oracle_job is not None:
        out["rel_l2_vs_oracle"] = guarded(oracle_job.compare, finals)
    if not args.no_serve:
        out["serving"] = guarded(run_serving, args)
        out["serving_saturated"] = guarded(run_serving_saturated, args)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def guarded(fn, *a):
    """A secondary measurement must not cost the main line."""
    try:
        return fn(*a)
    except Exception as e:   # noqa: BLE001
        return {"error": "%s: %s" % (type(e).__name__, e)}


def run_batch(args, stream, flush):
    """64 uneven simulations advanced together (grouped launches + graphs)."""
    import torch

    import paper_1911_08158_gb300 as ads
    from paper_1911_08158_gb300 import workloads as wl
    cases = wl.batch_cases(count=64, seed=0, steps=50)
    sims = []
    for c in cases:
        sim = ads.Simulation(c.n_elem, c.p, c.tau, precision="fp32", stream=stream)
        sim.set_gaussian_state(c.u0, None)
        sims.append(sim)
    tiles = [s.autotune(3) for s in sims]
    dof_steps = sum(dofs(s) for s in sims) * 50
    ads.batch_step(sims, 50)   # warm-up: first grouped step, graph capture
    torch.cuda.synchronize()
    reps = max(1, min(args.steps, 5))
    t = 0.0
    l0 = ads.launch_count()
    for _ in range(reps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ads.batch_step(sims, 50)
        e1.record(stream)
        e1.synchronize()
        t += e0.elapsed_time(e1) / 1e3
    launches_per_step = (ads.launch_count() - l0) / (reps * 50)
    n = sum(dofs(s) for s in sims)
    interior = sum((s.n[0] - 2) * (s.n[1] - 2) * (s.n[2] - 2) for s in sims)
    # kernel shares: each member's kernels timed by CUDA events in one profiled
    # step of its own (ads_profile_step), summed over the members
    kms = {}
    for s in sims:
        for name, ms in s.profile_step():
            kms[name] = kms.get(name, 0.0) + ms
    tot = sum(kms.values())
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    traffic = None   # ncu DRAM bytes per interior DOF-step of K1 + K3 on an L2-exceeding batch
    try:
        import glob
        for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
            for line in open(path):
                f = line.split()
                if len(f) == 3 and f[0] == "traffic_bytes_per_interior_dof_step" and f[1] == "batch":
                    traffic = float(f[2])
    except Exception:
        pass
    rate = interior * 50 * reps / t   # interior DOF-steps/s
    roof = {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": "measured" if peaks else "fallback",
            "state_bytes_per_interior_dof_step": 16,
            "achieved_state": round(rate * 16 / 1e9, 1), "frac_state": round(rate * 16 / 1e9 / peak, 4),
            "two_pass_bytes_per_interior_dof_step": 28,
            "achieved_two_pass": round(rate * 28 / 1e9, 1), "frac_two_pass": round(rate * 28 / 1e9 / peak, 4),
            "kernel_share": {k: round(v / tot, 4) for k, v in kms.items()},
            "traffic_bytes_per_interior_dof_step": traffic,
            "footprint_bytes": int(sum(s.device_bytes for s in sims))}
    for s in sims:
        s.close()
    return {"value": dof_steps * reps / t, "unit": UNIT, "simulations": len(cases), "steps_each": 50,
            "total_dofs": n, "interior_dofs": interior, "reps": reps, "ms_per_rep": t / reps * 1e3,
            "tiles_fused": sum(1 for s, r in zip(cases, tiles) if r == s.n_elem[1] + s.p - 2),
            "launches_per_step": launches_per_step, "roofline": roof,
            "workload": "batch64_pwave_uneven_32to160_p2p3_50steps_fp32"}


def run_elastic(args, stream, flush):
    """Elasticity (96^3 elements, p = 2, lambda = mu = rho = 1, tau = 2e-3,
    100 steps, seeded Gaussian velocity pulse): FP32 and FP64 paths, the
    FP32 displacement error against the FP64 path, and per-phase times."""
    import torch

    import paper_1911_08158_gb300 as ads
    from paper_1911_08158_gb300 import workloads as wl
    case = wl.elastic_case()
    out = {"workload": "elastic_96cubed_p2_100steps", "steps": case.steps}
    finals = {}
    for prec in ("fp32", "fp64"):
        sim = ads.Simulation(case.n_elem, case.p, case.tau, kind="elastic", lam=case.lam, mu=case.mu,
                             rho=case.rho, precision=prec, stream=stream)
        sim.set_gaussian_state(None, case.v0)
        sim.step(2)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(case.steps)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        dofs = int(np.prod(sim.n)) * 3
        out[prec] = {"value": dofs * case.steps / t, "unit": UNIT, "ms_per_step": t / case.steps * 1e3}
        if prec == "fp32":
            # the state alone: U^n and U^{n-1} read, U^{n+1} written once per
            # interior unknown and step (3 x 4 bytes); the fused schedule moves
            # more (13 launches a step)
            peak, src = hbm_peak()
            interior = int(np.prod([m - 2 for m in sim.n])) * 3
            ach = interior * case.steps / t * 12 / 1e9
            out["roofline"] = {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": src,
                               "state_bytes_per_interior_dof_step": 12, "achieved_state": round(ach, 1),
                               "frac_state": round(ach / peak, 4)}
        finals[prec] = sim.get_state(fields=("u",))[0]
        if prec == "fp32":
            out["phases_ms"] = {k: round(v, 4) for k, v in sim.profile_step()}
        sim.close()
    out["rel_l2_fp32_vs_fp64_u"] = float(np.linalg.norm(finals["fp32"] - finals["fp64"]) /
                                         np.linalg.norm(finals["fp64"]))
    return out


def run_serving(args):
    """The request stream of the serving configuration; with N ranks each GPU
    serves its shard of whole requests (no communication) and rank 0 reports
    its own latencies."""
    from paper_1911_08158_gb300 import workloads as wl
    from paper_1911_08158_gb300.serve import Server, shard_requests
    ws, rank, _ = dist_env()
    reqs = wl.serving_requests(count=args.serve_requests, rate=20.0, seed=0)
    mine = shard_requests(reqs, rank, ws)
    rep = Server(150 * 10 ** 9, precision="fp32", chunk=16).run(mine)
    out = rep.summary()
    out.update(workload="serving_poisson20_%dreq_wave80_elastic20_24to256_budget150GB_fp32" % len(reqs),
               unit_latency="s", shard="rank %d of %d: %d requests" % (rank, ws, len(mine)))
    return out


def run_serving_saturated(args):
    """The same 500 requests arriving 100x faster (2000 req/s: the whole
    stream within a quarter second) under a 4 GB budget: the device is busy
    throughout and admission waits on memory, so DOF-steps/s measures the
    device under contention and p50/p99 include the queueing."""
    from paper_1911_08158_gb300 import workloads as wl
    from paper_1911_08158_gb300.serve import Server, shard_requests
    ws, rank, _ = dist_env()
    budget = 4 * 10 ** 9
    reqs = wl.serving_requests(count=args.serve_requests, rate=2000.0, seed=0)
    mine = shard_requests(reqs, rank, ws)
    rep = Server(budget, precision="fp32", chunk=16).run(mine)
    out = rep.summary()
    out.update(workload="serving_poisson2000_%dreq_wave80_elastic20_24to256_budget4GB_fp32" % len(reqs),
               unit_latency="s", budget_bytes=budget, shard="rank %d of %d: %d requests" % (rank, ws, len(mine)))
    return out


class OracleRunner:
    """The FP64 CPU oracle on the benchmark workload (128^3 elements, one
    simulation per degree in PS), set up once (1D matrices, 3D source
    quadrature; not timed) and advanced one Newmark step at a time."""

    def __init__(self, degrees=PS):
        import oracle as ora
        from paper_1911_08158_gb300 import workloads as wl
        self.ora = ora
        self.sims = []
        for p in degrees:
            case = wl.ricker_case(ne=NE, p=p)
            s = ora.Space(case.n_elem, case.p)
            G = s.load_gauss(case.source["amp"], case.source["center"], case.source["den"])
            z = s.zeros()
            a = s.pwave_accel(z, 0.0, 1.0, G)
            self.sims.append(dict(s=s, G=G, tau=case.tau, state=(z, z, a), n=0, dofs=int(np.prod(s.n))))

    def run(self, seconds: float):
        """At least one step of every simulation, round robin, for `seconds`;
        returns (DOF-steps, steps, elapsed)."""
        done, steps, t = 0, 0, 0.0
        while steps < len(self.sims) or t < seconds:
            m = self.sims[steps % len(self.sims)]
            t0 = time.perf_counter()
            m["state"] = m["s"].pwave_run(*m["state"], m["tau"], 1, step0=m["n"], G=m["G"])
            t += time.perf_counter() - t0
            m["n"] += 1
            done += m["dofs"]
            steps += 1
        return done, steps, t

    def threads(self):
        return self.ora.num_threads()


class OracleFinals:
    """The benchmark workload run to its end by the FP64 CPU oracle (in a
    thread: the oracle's C loops release the interpreter), for the error of
    the GPU paths against it."""

    def __init__(self, degrees, steps):
        self.result, self.error = {}, None
        self.t = threading.Thread(target=self._run, args=(degrees, steps), daemon=True)
        self.t.start()

    def _run(self, degrees, steps):
        try:
            r = OracleRunner(degrees)
            for m in r.sims:
                u, v, a = m["s"].pwave_run(*m["state"], m["tau"], steps, step0=0, G=m["G"])
                self.result[m["s"].p] = m["s"].pad(u)
        except Exception as e:   # noqa: BLE001
            self.error = e

    def compare(self, finals):
        self.t.join()
        if self.error:
            raise self.error
        out = {"steps": NSTEPS}
        for p, (u64, u32) in finals.items():
            ref = self.result[p]
            nr = float(np.linalg.norm(ref))
            out["fp64_p%d" % p] = float(np.linalg.norm(u64 - ref) / nr)
            out["fp32_p%d" % p] = float(np.linalg.norm(u32 - ref) / nr)
        return out


def cpu_table(args):
    """The oracle timed per configuration at 1 thread and at all cores
    (bounded samples of Newmark steps; set-up not timed): DOF-steps/s."""
    import oracle as ora
    from paper_1911_08158_gb300 import workloads as wl
    allc = ora.num_threads()
    rows = []

    def time_wave(case, steps):
        s = ora.Space(case.n_elem, case.p)
        G = None
        if case.source:
            G = s.load_gauss(case.source["amp"], case.source["center"], case.source["den"])
        u = s.project_gauss(case.u0["amp"], case.u0["center"], case.u0["den"]) if case.u0 else s.zeros()
        z = s.zeros()
        a = s.pwave_accel(u, 0.0, 1.0, G)
        out = {}
        for th in (1, allc):
            ora.set_num_threads(th)
            t0 = time.perf_counter()
            s.pwave_run(u, z, a, case.tau, steps, step0=0, G=G)
            out[th] = (int(np.prod(s.n)) * steps / (time.perf_counter() - t0), steps)
        return out

    def time_elastic(case, steps):
        s = ora.Space(case.n_elem, case.p)
        g = s.project_gauss(case.v0["amp"], case.v0["center"], case.v0["den"])
        V0 = np.stack([case.v0["dir"][i] * g for i in range(3)])
        U0 = np.zeros_like(V0)
        Up = s.elastic_start(case.tau, case.lam, case.mu, case.rho, U0, V0)
        out = {}
        for th in (1, allc):
            ora.set_num_threads(th)
            t0 = time.perf_counter()
            s.elastic_run(case.tau, case.lam, case.mu, case.rho, steps, U0, Up, step0=0)
            out[th] = (3 * int(np.prod(s.n)) * steps / (time.perf_counter() - t0), steps)
        return out

    for name, fn, case, steps in (
            ("C1 16^3 p=2 FP64 pulse", time_wave, wl.pulse_case(ne=16, p=2, tau=1e-2, steps=20), 20),
            ("C2 128^3 p=2 Ricker", time_wave, wl.ricker_case(ne=NE, p=2), args.cpu_table_steps),
            ("C2 128^3 p=3 Ricker", time_wave, wl.ricker_case(ne=NE, p=3), args.cpu_table_steps),
            ("C3 96^3 p=2 elasticity", time_elastic, wl.elastic_case(), args.cpu_table_steps)):
        r = fn(case, steps)
        rows.append({"config": name, "threads_1": round(r[1][0]), "threads_all": round(r[allc][0]),
                     "steps_timed": steps, "cores": allc})
    ora.set_num_threads(allc)
    print(json.dumps({"cpu_table": rows, "unit": UNIT, "kind": "oracle", "cores": allc}))


def cpu_baseline(seconds: float):
    r = OracleRunner()
    dofs, n, t = r.run(seconds)
    return {"value": dofs / t, "unit": UNIT, "cores": r.threads(), "kind": "oracle",
            "sample": "%d Newmark steps of the 128^3 p=2 and p=3 simulations, alternating (FP64 oracle, "
                      "OpenMP over lines), %.1f s" % (n, t)}


def run_reference(args):
    """The reference arm: the CPU oracle (there is no reference implementation
    of the paper) on this benchmark's workload, metric and unit; each step is a
    bounded sample of Newmark steps of both simulations."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = max(1.0, args.cpu_seconds / max(args.steps, 1))
    r = OracleRunner()
    for _ in range(args.warmup):
        r.run(0.0)
    tt, dd, nn = 0.0, 0, 0
    for _ in range(args.steps):
        d, n, t = r.run(per_step)
        tt += t
        dd += d
        nn += n
    value = dd / tt
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "n_elem": NE, "p": list(PS), "tau": 2e-3,
                      "sample": "Newmark steps of both simulations, alternating, %.1f s per step" % per_step},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": r.threads(), "kind": "oracle",
                            "sample": "%d Newmark steps of the 128^3 p=2 and p=3 simulations in %.1f s" % (nn, tt)},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def profile_case(ne, p: int, steps: int, batch: int = 1, tune: int = 3, kind: str = "wave"):
    """Small fixed case for ncu captures: `batch` FP32 simulations of ne
    (n or nx,ny,nz) elements with autotuned K1 layouts (tune = 0: the first
    candidate, no timed trials), advanced together (grouped launches; no
    timing): two warm-up steps, then `steps` single steps.  kind 'elastic':
    one elasticity simulation (lambda = mu = rho = 1, seeded velocity pulse)."""
    import torch

    import paper_1911_08158_gb300 as ads
    from paper_1911_08158_gb300 import workloads as wl

    torch.cuda.set_device(0)
    if kind == "batch64":
        # the 64-simulation batch (1.1 GB): 2 warm-up grouped steps, then `steps`
        cases = wl.batch_cases(count=64, seed=0, steps=50)
        sims = []
        for c in cases:
            sim = ads.Simulation(c.n_elem, c.p, c.tau, precision="fp32")
            sim.set_gaussian_state(c.u0, None)
            sim.autotune(tune)
            sims.append(sim)
        ads.batch_step(sims, 2)
        for _ in range(steps):
            ads.batch_step(sims, 1)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "batch64", "steps": steps, "tune": tune,
                          "device_bytes": sum(s.device_bytes for s in sims)}))
        return
    if kind == "elastic":
        c = wl.elastic_case(ne=ne, p=p)
        sim = ads.Simulation(c.n_elem, c.p, c.tau, kind="elastic", lam=c.lam, mu=c.mu, rho=c.rho, precision="fp32")
        sim.set_gaussian_state(None, c.v0)
        sim.step(2)
        for _ in range(steps):
            sim.step(1)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": ne, "p": p, "kind": kind, "steps": steps, "device_bytes": sim.device_bytes}))
        return
    sims = []
    for i in range(batch):
        case = wl.ricker_case(ne=ne, p=p, seed=i)
        sim = ads.Simulation(case.n_elem, case.p, case.tau, precision="fp32")
        sim.set_source(case.source)
        sim.set_gaussian_state(None, None)
        sim.autotune(tune)   # the layout the benchmark would use (tune = 3)
        sims.append(sim)
    ads.batch_step(sims, 2)
    for _ in range(steps):
        ads.batch_step(sims, 1)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": ne, "p": p, "steps": steps, "batch": batch,
                      "device_bytes": sum(s.device_bytes for s in sims)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-simulation batch measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-elastic", action="store_true", help="skip the elasticity measurement")
    ap.add_argument("--serve-requests", type=int, default=500)
    ap.add_argument("--no-peaks", action="store_true", help="skip the CUDA-core FMA peak measurement")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the error of the 200-step runs against the CPU oracle")
    ap.add_argument("--cpu-table", action="store_true",
                    help="time the CPU oracle per configuration at 1 thread and all cores, print, exit")
    ap.add_argument("--cpu-table-steps", type=int, default=4)
    ap.add_argument("--autotune-steps", type=int, default=3,
                    help="trial steps per K1 layout candidate (0: take the first candidate)")
    ap.add_argument("--profile-case", default="", help="run a small case (n or nx,ny,nz elements) for ncu and exit")
    ap.add_argument("--profile-p", type=int, default=2)
    ap.add_argument("--profile-batch", type=int, default=1, help="simulations advanced together in the profile case")
    ap.add_argument("--profile-tune", type=int, default=3, help="autotuner trial steps in the profile case")
    ap.add_argument("--profile-kind", default="wave", choices=["wave", "elastic", "batch64"])
    args = ap.parse_args()
    if args.cpu_table:
        cpu_table(args)
    elif args.profile_case:
        ne = tuple(int(v) for v in args.profile_case.split(",")) if args.profile_kind != "batch64" else (0,)
        profile_case(ne[0] if len(ne) == 1 else ne, args.profile_p, 4, args.profile_batch, args.profile_tune,
                     args.profile_kind)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
