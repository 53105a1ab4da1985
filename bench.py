"""Benchmark of the DVM transport hot path on one GB300 (replicas on N GPUs).

Workload (one step = one check interval of the source iteration, Sec. 3.1: 100 iterations of
sweep + quadrature + wall/source update, then the permeability and Err check of Eq. 15):
  2D random porous medium, 512 x 512 overlapping discs (seed 0, radii uniform in [6, 20] cells,
  solid fraction 0.5, periodic, non-percolating fluid filled), 32 x 32 half-range Gauss-Hermite
  velocities (1024), the Knudsen sweep {0.01, 0.1, 1, 10} as one batched context, FP32 h and
  moments, FP64 wall sums, G_p and Err.
Metric: cell-velocity updates per second = (fluid cells) x (velocities) x (iterations) x (problems)
/ time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the reference arm of this build) on the host cores.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KNS = [0.01, 0.1, 1.0, 10.0]
N_AXIS = 32
SIDE = 512
ITERS_PER_STEP = 100
METRIC = "cell·velocity updates/s"
WORKLOAD = ("2D random discs 512x512 (seed 0, r 6-20, solid fraction 0.5, periodic, percolating), "
            "32x32 Gauss-Hermite velocities, Kn {0.01,0.1,1,10} batched, FP32")
# algorithmic work of one cell-velocity update of the sweep (2D): source 2 FMA, upwind terms
# 2 x (2 FMA) + 2 FMA, one multiply by the reciprocal denominator, quadrature 3 MUL + 3 ADD
FLOPS_PER_UPDATE = 2 * 2 + 6 * 2 + 1 + 3 + 3
SMS, FP32_LANES_PER_SM = 152, 128


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench_%d.csv" % gpu_index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        load = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_replicas(local_ms, units_per_rank, device=None):
    """Whole-job throughput of independent replicas: every rank processed units_per_rank units in
    local_ms; the job time is the maximum over ranks and the value is the units of all ranks / that
    time.  Returns (value per second, max ms, world size).  Works with any torch.distributed
    backend (NCCL on GPUs, gloo on CPU) or without an initialised process group."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_per_rank)], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    return float(u.item()) / (ms_max * 1e-3), ms_max, ws


def _workload():
    from paper_1712_01132_gb300 import inputs
    mask = inputs.random_discs(SIDE, SIDE, seed=0)
    return mask, int((~mask).sum())


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1712_01132_gb300 import dvm

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    mask, nf = _workload()
    v, w = dvm.dvm_gh_velocity_grid(2, N_AXIS)
    nv = len(w)
    updates_per_step = nf * nv * ITERS_PER_STEP * len(KNS)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- device-resident timing: inputs already in HBM
    s = dvm.Solver([mask] * len(KNS), KNS, v, w, precision="fp32", lateral="periodic")
    for _ in range(args.warmup):
        s.iterate(ITERS_PER_STEP, 0.0)
    s.profile_enable(True)
    s.profile_read()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s.iterate(ITERS_PER_STEP, 0.0)          # 100 iterations + the Err check (host sync)
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms_total = e0.elapsed_time(e1)
    sweep_ms, sweep_n, fin_ms, fin_n = s.profile_read()
    s.profile_enable(False)
    ks = [s.permeability(b)[0] for b in range(len(KNS))]
    s.close()
    value, ms_max, _ = aggregate_replicas(ms_total, updates_per_step * args.steps, device="cuda")

    # ---------------- end to end through the public API with host buffers
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    h0 = torch.cuda.Event(enable_timing=True)
    h1 = torch.cuda.Event(enable_timing=True)
    h2d = d2h = 0
    h0.record(stream)
    for _ in range(e2e_steps):
        se = dvm.Solver([mask] * len(KNS), KNS, v, w, precision="fp32", lateral="periodic")
        se.iterate(ITERS_PER_STEP, 0.0)
        for b in range(len(KNS)):
            se.moments(b)
            se.permeability(b)
        hb, db = se.transfer_bytes()
        h2d += hb
        d2h += db
        se.close()
    h1.record(stream)
    barrier()
    e2e_ms = h0.elapsed_time(h1)
    e2e_value = updates_per_step * e2e_steps * ws / (e2e_ms * 1e-3)

    # ---------------- roofline of the dominant kernel (sweep), FP32 ALU bound
    peaks = _peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    peak_tflops = SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    per_launch_updates = nf * nv * len(KNS)
    sweep_avg_s = (sweep_ms / max(sweep_n, 1)) * 1e-3
    achieved = per_launch_updates * FLOPS_PER_UPDATE / sweep_avg_s / 1e12
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_tflops, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak_tflops, 4), "traffic": None,
                "kernel": "dvm::sweep2d_kernel<float,16>", "avg_launch_ms": round(sweep_avg_s * 1e3, 4),
                "share_of_step": round(sweep_ms / max(sweep_ms + fin_ms, 1e-9), 4),
                "peak_basis": "FP32 FMA issue, 152 SMs x 128 lanes x 2 flop x %.0f MHz (derived)" % sm_max,
                "flops_per_update": FLOPS_PER_UPDATE}

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "fluid_cells": nf, "velocities": nv, "problems": len(KNS),
                       "iterations_per_step": ITERS_PER_STEP,
                       "step": "100 source iterations (sweep+quadrature+finalize) + permeability/Err check",
                       "l2": "working set per iteration > L2 (band edge buffers ~0.5 GB, moments 50 MB)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "e2e": {"value": e2e_value, "unit": "updates/s", "h2d_bytes_per_step": int(h2d // e2e_steps),
                    "d2h_bytes_per_step": int(d2h // e2e_steps),
                    "includes": "context creation from host masks, 100 iterations, moment and permeability readout"},
            "gpu_launches": int(2 * ITERS_PER_STEP * args.steps),
            "roofline": roofline,
            "clocks": clocks,
            "permeability": dict(zip([str(k) for k in KNS], ks)),
        }
    if ws > 1:
        dist.destroy_process_group()
    return out


def cpu_baseline_sample(iters=1, kn=0.1):
    """The oracle as it stands, on the host cores, on a bounded sample: `iters` iterations of one
    Knudsen number of the same 512x512, 1024-velocity problem."""
    import oracle
    mask, nf = _workload()
    v, w = oracle.velocity_grid(2, N_AXIS)
    o = oracle.Oracle(mask, kn, v, w, lateral="periodic")
    t0 = time.perf_counter()
    o.iterate(iters)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": nf * len(w) * iters / dt, "unit": "updates/s", "cores": cores, "kind": "oracle",
            "sample": "%d FP64 oracle iteration(s) of the Kn=%g problem (512x512, 1024 velocities), %.1f s"
                      % (iters, kn, dt)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    import oracle
    mask, nf = _workload()
    v, w = oracle.velocity_grid(2, N_AXIS)
    o = oracle.Oracle(mask, 0.1, v, w, lateral="periodic")
    for _ in range(args.warmup):
        o.iterate(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.iterate(1)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    value = nf * len(w) * args.steps / dt
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "fluid_cells": nf, "velocities": len(w),
                       "step": "one FP64 oracle iteration of the Kn=0.1 problem (bounded sample of the workload)"},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": "%d oracle iterations, Kn=0.1, 512x512, 1024 velocities" % args.steps},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    else:
        out = run_gpu(args)
        if out is not None and not args.no_cpu_baseline and args.gpus == 1:
            out["cpu_baseline"] = cpu_baseline_sample()
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
