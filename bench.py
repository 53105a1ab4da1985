"""Benchmark of the DVM transport hot path on one GB300 (replicas on N GPUs).

One step = one check interval of the source iteration (Sec. 3.1): 100 iterations of sweep +
quadrature + wall/source update, then the permeability and the Err check of Eq. 15.
Metric: cell-velocity updates per second = (fluid cells) x (velocities) x (iterations) / time,
summed over the problems of the batch; config.full_grid_updates_per_s counts every grid cell.

Workloads (--workload):
  rock_128      (default) 3D Gaussian-field rock 128^3 (seed 0, correlation length 8, porosity 0.35,
                percolating cluster), 16^3 = 4096 velocities, Kn = 0.5, FP32: the largest
                configuration that runs on one GPU.
  kn_sweep_512  2D random porous medium, 512 x 512 overlapping discs (seed 0, radii uniform
                in [6, 20] cells, solid fraction 0.5, periodic, non-percolating fluid filled),
                32 x 32 half-range Gauss-Hermite velocities (1024), Kn in {0.01, 0.1, 1, 10} as one
                batched context; FP32 h and moments, FP64 wall sums, G_p and Err.
  disc_batch_64 64 seeded disc packings (seeds from 1000, sides uniform in 64..512, porosity
                0.4-0.7, radii 6-20, Kn log-uniform in [0.01, 10]) in one batched context,
                24 x 24 velocities, FP32.
Tile shapes are chosen by the library's autotuner before the timed region.  The timed steps run
the production loop: dvm_iterate with the CUDA-graph replay of each 100-iteration run; the graph
carries event-record nodes around every sweep and finalize launch, from which the roofline's
per-launch kernel time is read (same stream, same timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores (the reference arm).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ITERS_PER_STEP = 100
METRIC = "cell·velocity updates/s"
FP32_LANES_PER_SM = 128      # FP32 FMA lanes per SM on sm_100-family GPUs

WORKLOADS = {
    "kn_sweep_512": {
        "dims": 2, "n_axis": 32,
        "desc": "2D random discs 512x512 (seed 0, r 6-20, solid fraction 0.5, periodic, percolating), "
                "32x32 Gauss-Hermite velocities, Kn {0.01,0.1,1,10} batched, FP32",
        # source 2 FMA, upwind 2 x (2 FMA) + 2 FMA, reciprocal 1 MUL, quadrature 3 MUL + 3 ADD
        "flops_per_update": 2 * 2 + 6 * 2 + 1 + 3 + 3,
        "kernel": "dvm::sweep2d_f32x2_kernel<T1,0,0>",
        "l2": "working set per iteration > L2 (band edges and ghosts ~0.6 GB, moment partials 13 MB)",
    },
    "disc_batch_64": {
        "dims": 2, "n_axis": 24,
        "desc": "64 disc packings (seeds 1000+, sides 64-512, porosity 0.4-0.7, r 6-20, "
                "Kn log-uniform [0.01,10]) batched, 24x24 Gauss-Hermite velocities, FP32",
        "flops_per_update": 2 * 2 + 6 * 2 + 1 + 3 + 3,
        "kernel": "dvm::sweep2d_f32x2_kernel<T1,0,0>",
        "l2": "working set per iteration > L2 (band edges and ghosts of 64 problems ~2 GB)",
    },
    "rock_128": {
        "dims": 3, "n_axis": 16,
        "desc": "3D Gaussian-field rock 128^3 (seed 0, correlation length 8, porosity 0.35, percolating), "
                "16^3 Gauss-Hermite velocities, Kn 0.5, FP32",
        # source 3 FMA, upwind 3 x (2 FMA) + 3 FMA, reciprocal 1 MUL, quadrature 4 MUL + 4 ADD
        "flops_per_update": 3 * 2 + 9 * 2 + 1 + 4 + 4,
        "kernel": "dvm::sweep3d_f32x2_kernel<T1,0,0,0,0>",
        "l2": "working set per iteration > L2 (pencil edges and ghosts ~6 GB)",
    },
}


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


# workload -> (committed ncu summary holding the sweep's DRAM bytes per launch, kernel sources it was
# taken with)
TRAFFIC_PROFILES = {
    "kn_sweep_512": ("sweep2d_f32x2_kn_sweep_512.md", ("paper_1712_01132_gb300/csrc/sweep2d_f32x2.cu",
                                                       "paper_1712_01132_gb300/csrc/dvm_device.cuh",
                                                       "paper_1712_01132_gb300/csrc/dvm_internal.h")),
    "rock_128": ("sweep3d_f32x2_rock_128_launches.md", ("paper_1712_01132_gb300/csrc/sweep3d_f32x2.cu",
                                                        "paper_1712_01132_gb300/csrc/dvm_device.cuh",
                                                        "paper_1712_01132_gb300/csrc/dvm_internal.h")),
}


def measured_traffic(workload, tiles):
    """DRAM bytes per sweep launch from the committed ncu summary of the workload, or None when there
    is none, the tile shape differs or the kernel sources changed since the capture."""
    import hashlib
    if workload not in TRAFFIC_PROFILES:
        return None
    fname, sources = TRAFFIC_PROFILES[workload]
    try:
        text = open(os.path.join(ROOT, "profiles", fname)).read()
        fields = dict(line.split(": ", 1) for line in text.splitlines() if line.startswith("traffic_"))
        h = hashlib.sha256()
        for f in sources:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        if fields.get("traffic_source_sha256") != h.hexdigest():
            return None
        if fields.get("traffic_tiles") != " ".join(str(int(x)) for x in tiles):
            return None
        return int(fields["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


HBM_FALLBACK_GBS = 6800.0   # one earlier copy-bandwidth measurement on a GB300


def hbm_fractions(peaks, dims, cells, sweep_s, iter_s, traffic):
    """The path against the HBM roofline, next to the ALU one.  The method keeps no bulk h between
    iterations (Sec. 3.1): per iteration and grid cell it must read a code byte and d + 1 FP64
    moments and write 2^d (d + 1) FP32 quadrant/octant moment partials, 1 + 8 (d + 1) + 4 (d + 1) 2^d
    bytes, over the time of the iteration's sweep and finalize.  `traffic` is the measured DRAM bytes
    of one sweep launch (or None), over the sweep's own time."""
    peak = float(peaks.get("hbm_gbs") or HBM_FALLBACK_GBS)
    per_cell = 1 + 8 * (dims + 1) + 4 * (dims + 1) * 2 ** dims
    alg = per_cell * cells
    alg_gbs = alg / iter_s / 1e9
    out = {"peak_gbs": peak,
           "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)" if peaks.get("hbm_gbs")
                         else "fallback 6.8 TB/s",
           "algorithmic_bytes_per_cell": per_cell,
           "algorithmic_bytes_per_iteration": alg,
           "algorithmic_gbs": round(alg_gbs, 1),
           "algorithmic_frac": round(alg_gbs / peak, 5),
           "dram_gbs": None, "dram_frac": None}
    if traffic:
        dram_gbs = traffic / sweep_s / 1e9
        out["dram_gbs"] = round(dram_gbs, 1)
        out["dram_frac"] = round(dram_gbs / peak, 4)
    return out


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, directory=None):
        import tempfile
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(directory or tempfile.gettempdir(), "clocks_bench_%d.csv" % gpu_index)

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
        with open(self.path) as f:
            return parse_clocks(f)


def parse_clocks(lines):
    """Summary of `nvidia-smi --query-gpu=ClockSampler.FIELDS --format=csv,noheader,nounits` lines:
    the median SM clock over the samples under load (above half the maximum clock; all samples if
    none is), the maximum SM clock, and the throttle reasons seen active in any sample."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
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


def problems(name, side=128):
    """(masks, Knudsen numbers, fluid cells per problem) of a workload (side: rock edge length)."""
    from paper_1712_01132_gb300 import inputs
    if name == "kn_sweep_512":
        mask = inputs.random_discs(512, 512, seed=0)
        kns = [0.01, 0.1, 1.0, 10.0]
        masks = [mask] * len(kns)
    elif name == "disc_batch_64":
        batch = inputs.disc_batch(64, seed0=1000)
        masks, kns = [b[0] for b in batch], [b[1] for b in batch]
    elif name == "rock_128":
        masks, kns = [inputs.gaussian_rock(side, seed=0, corr_len=8.0, porosity=0.35)], [0.5]
    else:
        raise ValueError(name)
    return masks, kns, [int((~m).sum()) for m in masks]


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1712_01132_gb300 import dvm

    W = WORKLOADS[args.workload]
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    masks, kns, nfs = problems(args.workload, args.side)
    v, w = dvm.dvm_gh_velocity_grid(W["dims"], W["n_axis"])
    nv = len(w)
    updates_per_iter = sum(nfs) * nv
    updates_per_step = updates_per_iter * ITERS_PER_STEP
    stream = torch.cuda.current_stream()
    base = dict(precision="fp32", lateral="periodic")

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- tile shape from the autotuner (untimed setup)
    tune = dvm.autotune(masks, kns, v, w, iters=5 if W["dims"] == 2 else 2, **base)
    t1, rows, tune_ms = tune.tile_x1, tune.band_rows, tune.ms
    opts = dict(base, tile_x1=t1, band_rows=rows, group_warps=tune.group_warps, use_graph=True)

    # ---------------- device-resident timing: inputs already in HBM
    s = dvm.Solver(masks, kns, v, w, **opts)
    s.profile_enable(True)                      # event nodes inside the captured graphs
    for _ in range(args.warmup):                # (the first step captures the graph)
        s.iterate(ITERS_PER_STEP, 0.0)
    s.profile_read()
    sampler = ClockSampler(local, args.clocks_dir)
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
    ks = [s.permeability(b)[0] for b in range(len(masks))]
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
        se = dvm.Solver(masks, kns, v, w, **opts)
        se.iterate(ITERS_PER_STEP, 0.0)
        for b in range(len(masks)):
            se.moments(b)
            se.permeability(b)
        hb, db = se.transfer_bytes()
        h2d += hb
        d2h += db
        se.close()
    h1.record(stream)
    barrier()
    e2e_ms = h0.elapsed_time(h1)
    e2e_value, _, _ = aggregate_replicas(e2e_ms, updates_per_step * e2e_steps, device="cuda")

    # ---------------- roofline of the dominant kernel (sweep), FP32 ALU bound
    peaks = _peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    fma_measured = dvm.alu_peak("fp32")          # microbenchmark cross-check of the derived peak
    sweep_avg_s = (sweep_ms / max(sweep_n, 1)) * 1e-3
    achieved = updates_per_iter * W["flops_per_update"] / sweep_avg_s / 1e12
    kernel = W["kernel"].replace("T1", str(t1))
    traffic = measured_traffic(args.workload if args.side == 128 else "",
                               (t1, rows, tune.group_warps) if W["dims"] == 3 else (t1, rows))
    hbm = hbm_fractions(peaks, W["dims"], int(sum(m.size for m in masks)), sweep_avg_s,
                        ((sweep_ms + fin_ms) / max(sweep_n, 1)) * 1e-3, traffic)
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_tflops, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak_tflops, 4),
                "traffic": traffic,
                "kernel": kernel, "avg_launch_ms": round(sweep_avg_s * 1e3, 4),
                "share_of_step": round(sweep_ms / max(sweep_ms + fin_ms, 1e-9), 4),
                "peak_basis": "FP32 FMA issue, %d SMs x 128 lanes x 2 flop x %.0f MHz (SM count from the "
                              "device, max SM clock measured in MEASURED_PEAKS.json)" % (sms, sm_max),
                "timing": "CUDA events recorded by the captured graph around every sweep launch, "
                          "summed over the timed steps",
                "peak_fma_microbenchmark": round(fma_measured, 2),
                "flops_per_update": W["flops_per_update"], "updates_per_launch": updates_per_iter,
                "hbm": hbm}

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload if args.side == 128 else "%s_side%d" % (args.workload, args.side),
                       "description": W["desc"], "fluid_cells": sum(nfs),
                       "grid_cells": int(sum(m.size for m in masks)),
                       "full_grid_updates_per_s": value * sum(m.size for m in masks) / max(sum(nfs), 1),
                       "velocities": nv, "problems": len(masks), "iterations_per_step": ITERS_PER_STEP,
                       "step": "100 source iterations (sweep+quadrature+finalize) + permeability/Err check",
                       "tiles": {"tile_x1": t1, "band_rows": rows, "group_warps": tune.group_warps,
                                 "autotuned_ms_per_iteration": round(tune_ms, 4)},
                       "l2": W["l2"],
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "e2e": {"value": e2e_value, "unit": "updates/s", "h2d_bytes_per_step": int(h2d // e2e_steps),
                    "d2h_bytes_per_step": int(d2h // e2e_steps),
                    "includes": "context creation from host masks, 100 iterations, moment and permeability readout"},
            "gpu_launches": int(2 * ITERS_PER_STEP * args.steps),
            "roofline": roofline,
            "clocks": clocks,
            "permeability": [float(k) for k in ks] if len(ks) > 8 else dict(zip([str(k) for k in kns], ks)),
        }
    if rank == 0 and ws == 1 and args.workload == "rock_128" and not args.no_time_to_tol:
        out["config"]["time_to_tolerance"] = time_to_tolerance_section(args, opts)
    if ws > 1:
        dist.destroy_process_group()
    return out


def time_to_tolerance_section(args, opts):
    """The metric's second part on the learned-warm-start configuration: a 3D U-Net trained in this
    run by the library's kernels on solver runs of seeded 64^3 rocks (Kn log-uniform in [0.05, 5]),
    then on the held-out 128^3 rock (seed 10000, Kn 0.5) the iterations and wall time to Err < 1e-6
    of the plain FP32, plain FP64 and network-warm FP32 starts, each with its true k error."""
    import time
    import torch
    from paper_1712_01132_gb300 import inputs, warmstart
    t0 = time.perf_counter()
    data, t_data = warmstart.training_set(args.ttt_train, side=64, nv=16, log=lambda *a: None)
    net, info = warmstart.train_network(data, levels=args.ttt_levels, base=args.ttt_base, steps=args.ttt_steps,
                                        lr=5e-4, constant_lr=True, log=lambda *a: None)
    del data
    mask = inputs.gaussian_rock(128, seed=10000, corr_len=8.0, porosity=0.35)
    fp32 = {k: opts[k] for k in ("tile_x1", "band_rows", "group_warps")}
    res = warmstart.time_to_tolerance(mask, 0.5, 16, net=net, tol=1e-6, ref_tol=1e-8, fp64=True, max_iter=3000,
                                      fp32_options=fp32)
    torch.cuda.synchronize()
    res.update({"geometry": "gaussian_rock(128, seed=10000, corr_len=8, porosity=0.35), held out",
                "network": dict(info, train_runs=args.ttt_train, train_side=64, data_seconds=round(t_data, 1)),
                "section_seconds": round(time.perf_counter() - t0, 1)})
    return res


def _oracle_sample(name, budget_iters=None):
    """A bounded sample of the workload for the oracle: (list of (mask, kn), iterations, text)."""
    masks, kns, nfs = problems(name)
    if name == "kn_sweep_512":
        it = budget_iters or 25
        return [(masks[1], kns[1])], it, "%d FP64 oracle iterations of the Kn=0.1 problem (512x512, 1024 velocities)" % it
    if name == "disc_batch_64":
        it = budget_iters or 2
        return list(zip(masks, kns)), it, "%d FP64 oracle iteration(s) of each of the 64 problems (576 velocities)" % it
    it = budget_iters or 1
    return [(masks[0], kns[0])], it, "%d FP64 oracle iteration(s) of the 128^3 rock (4096 velocities)" % it


def _time_oracle(sample, iters, dims, n_axis):
    import oracle
    v, w = oracle.velocity_grid(dims, n_axis)
    units, dt = 0, 0.0
    for mask, kn in sample:
        o = oracle.Oracle(mask, kn, v, w, lateral="periodic")
        t0 = time.perf_counter()
        o.iterate(iters)
        dt += time.perf_counter() - t0
        units += int((~mask).sum()) * len(w) * iters
        del o
    return units, dt


def cpu_baseline_sample(name):
    """The oracle as it stands, on the host cores, on a bounded sample of the same workload."""
    W = WORKLOADS[name]
    sample, iters, text = _oracle_sample(name)
    units, dt = _time_oracle(sample, iters, W["dims"], W["n_axis"])
    return {"value": units / dt, "unit": "updates/s", "cores": _cores(), "kind": "oracle",
            "sample": "%s, %.1f s" % (text, dt)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    W = WORKLOADS[args.workload]
    sample, _, _ = _oracle_sample(args.workload, budget_iters=1)
    if args.workload == "disc_batch_64":
        sample = sample[:8]                       # a bounded slice of the batch per step
    if args.workload == "rock_128":
        # a slab of the rock (its first 16 x3 planes, all 4096 velocities) per step: one iteration
        # of the whole rock takes ~16 s on 16 cores, too long for K + W steps
        sample = [(sample[0][0][:16], sample[0][1])]
    for _ in range(args.warmup):
        _time_oracle(sample[:1], 1, W["dims"], W["n_axis"])
    units, dt = 0, 0.0
    for _ in range(args.steps):
        u, d = _time_oracle(sample, 1, W["dims"], W["n_axis"])
        units += u
        dt += d
    value = units / dt
    text = "per step one FP64 oracle iteration of %s" % (
        "the Kn=0.1 problem" if args.workload == "kn_sweep_512" else
        "problems 0-7 of the batch" if args.workload == "disc_batch_64" else
        "a 128 x 128 x 16 slab (x3 planes 0-15) of the 128^3 rock, 4096 velocities")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": W["desc"],
                       "step": text + " (bounded sample of the workload)"},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": _cores(), "kind": "oracle",
                             "sample": "%d steps: %s" % (args.steps, text)},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rock_128", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the raw nvidia-smi clock samples (default: the temp directory)")
    ap.add_argument("--side", type=int, default=128,
                    help="edge length of the rock_128 geometry (smaller only for profiling captures)")
    ap.add_argument("--no-time-to-tol", action="store_true",
                    help="skip the time-to-tolerance section (plain FP32 / FP64 / warm FP32 starts)")
    ap.add_argument("--ttt-train", type=int, default=32, help="solver runs in the in-run training set")
    ap.add_argument("--ttt-steps", type=int, default=1500, help="training steps of the in-run network")
    ap.add_argument("--ttt-levels", type=int, default=4)
    ap.add_argument("--ttt-base", type=int, default=32)
    args = ap.parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    else:
        out = run_gpu(args)
        if out is not None and not args.no_cpu_baseline and out["n_gpus"] == 1:
            out["cpu_baseline"] = cpu_baseline_sample(args.workload)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
