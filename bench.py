#!/usr/bin/env python
"""Benchmark of the COSEnu RK4-stage engine on GB300.

Workload (the roofline run): nz = 2^20 z cells, nv = 256 v bins, both species,
4 real components each; z in [-25600, 25600) (dz = 0.048828125), dt = 0.4 dz,
mu = 10, omega = 0, alpha = 0.9, sigma_nu = 0.6, sigma_nubar = 0.5, random-phase
off-diagonal seed 1e-6 (splitmix64, seed 12866).  A step is one full RK4 step
(four fused stage kernels) over the whole grid.  Metric: cell-updates/s, a cell
being one (z, v, species) triple advanced by one RK4 step.

Default arm: the CUDA library through its C ABI, mixed precision, FD4 + KO.
The line also carries the other three (scheme, precision) variants, the
roofline of the dominant stage kernel, an end-to-end figure through the C ABI
with host buffers, the oracle timed on the host cores, and clocks sampled
during the timed region.

--impl reference: the FP64 CPU oracle on a z-slab sample of the same workload.

Several GPUs (torchrun): independent replicas, one per rank (the workload is
one periodic grid per GPU; no data crosses GPUs), timed with a barrier and the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NZ, NV = 1 << 20, 256
DZ = 3200.0 / 65536.0
L = NZ * DZ
NZ_FULL = NZ
MU, ALPHA, SIG_NU, SIG_NUBAR, EPS0, SEED = 10.0, 0.9, 0.6, 0.5, 1e-6, 12866
WORKLOAD = ("roofline run: nz=2^20, nv=256, z in [-25600,25600), dt=0.4 dz, mu=10, omega=0, "
            "alpha=0.9, sigma=(0.6,0.5), random-phase seed 1e-6")

# Algorithmic HBM bytes per real component per launch of each kernel of an RK4
# step (k = 1..4 the fused stage kernels, k = 5 the increment kernel).
# fp64 (all arrays double): stage 1 reads y, writes d1; stage s = 2..4 reads y,
#   d_{s-1}, writes d_s; the increment kernel reads y, d1..d4 and writes the new
#   y into the other state buffer.
# mixed (state y double plus its float copy y32; increments float): stages 1-4
#   read y32 instead of y; the increment kernel reads y, d1..d4 and writes y,
#   y32 in place.
STAGE_BYTES = {"fp64": (16, 24, 24, 24, 48), "mixed": (8, 12, 12, 12, 36)}
KERNEL_NAMES = ("stage 1", "stage 2", "stage 3", "stage 4", "increment")
# FP64 flops per cell (4 reals) per launch of the fp64 kernels, counted from the
# kernels' arithmetic (FMA = 2 flops, a reciprocal = 1): stage input y + delta 4
# (stages 2-4), v-moment partials with the warp reduction 18 (FD4+KO, two
# columns per thread) or 22 (WENO7, one; the species sign is the reducer's),
# Hamiltonian 6 (one FMA per component from the reducer's coefficients, which
# carry the stage factor), commutator 11, advection 40 (FD4+KO: one FMA per
# window row, the two stencils combined, the stage factor in the weights) or
# 480 (WENO7: 117 per face for the reconstruction in differences, 3 for the
# flux difference); the increment kernel 32 (four FMA per real).
FP64_FLOPS_PER_CELL = {"fdko": (75, 79, 79, 79, 32), "weno7": (519, 523, 523, 523, 32)}
SCHEMES = {"fdko": 0, "weno7": 1}
PRECS = {"fp64": 0, "mixed": 1}
SMS = 152  # streaming multiprocessors of a GB300
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy bandwidth is the peak used)


def fp64_peak():
    """FP64 FMA peak measured by the FMA probe (profiles/fma_peak.json), else the
    unit-count figure 152 SMs x 2 FP64 FMA lanes x 2 flops x 2.07 GHz."""
    path = os.path.join(ROOT, "profiles", "fma_peak.json")
    if os.path.exists(path):
        return float(json.load(open(path))["fp64_tflops"]), "measured (FMA probe)"
    return 152 * 2 * 2 * 2.07e9 / 1e12, "unit counts"


FP64_PEAK_TFLOPS, FP64_PEAK_KIND = fp64_peak()


def kernel_counts(key):
    """Per-cell instruction counts of the compiled kernels measured by ncu
    (profiles/kernel_counts.json): "fp64_pipe_lane_ops_per_cell" (FP64-pipe lane
    operations of each kernel of an FP64 step; every FP64 instruction occupies the pipe
    as long as an FMA, so the pipe's limit is the FMA probe's rate in lane-operations,
    peak TFLOP/s / 2) or "warp_inst_per_cell" (warp instructions of the mixed WENO7
    stage kernels, against the issue limit of 4 per SM and clock).  None if absent or
    taken on different source."""
    path = os.path.join(ROOT, "profiles", "kernel_counts.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get(key)


def fp64_pipe_ops():
    return kernel_counts("fp64_pipe_lane_ops_per_cell")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ ncu traffic


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("stage_kernel.cuh", "stage_body.inc", "cosenu_device.cuh", "diag_kernels.cu",
              "diag_kernels.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2203_12866_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(scheme, prec, stage):
    """DRAM bytes per launch of the stage kernel from the committed ncu summary,
    scaled to this workload; None when absent or taken on different source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("source_hash") != kernel_source_hash():
        return None
    rec = d.get("kernels", {}).get(f"{scheme}_{prec}_stage{stage}")
    if not rec:
        return None
    return rec["dram_bytes_per_launch"] * (8 * NZ * NV) / rec["reals_per_launch"]


# ------------------------------------------------------------------ distributed


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        if args.impl == "reference":
            dist.init_process_group("gloo")
        else:
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
    return world, rank, local


def dist_max(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ------------------------------------------------------------------ oracle arm


def oracle_rate(rows, steps, scheme="fdko"):
    """Cell-updates/s of the FP64 oracle on a periodic z-slab of `rows` rows of the
    workload (same dz, nv, parameters); returns (rate, seconds, threads)."""
    import oracle
    from paper_2203_12866_gb300 import inputs
    oracle.build()
    u0 = inputs.collective_rows(range(rows), NV, alpha=ALPHA, sigma_nu=SIG_NU,
                                sigma_nubar=SIG_NUBAR, eps0=EPS0, seed=SEED)
    p = oracle.params(rows, NV, rows * DZ, SCHEMES[scheme], mu=MU, cfl=0.4)
    t0 = time.perf_counter()
    oracle.step(p, u0, steps)
    dt = time.perf_counter() - t0
    return 2 * rows * NV * steps / dt, dt, oracle.num_threads()


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    rows = args.cpu_rows
    oracle_rate(min(rows, 256), 1)  # build, page in
    for _ in range(args.warmup):
        oracle_rate(rows, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rate(rows, 1)
    sec = time.perf_counter() - t0
    value = 2 * rows * NV * args.steps / sec
    sample = f"z-slab of {rows} rows x nv=256 x 2 species (periodic, same dz and parameters), FD+KO"
    line = {
        "impl": "reference", "metric": "cell-updates/s (z*v*species per RK4 step)",
        "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "scheme": "FD+KO", "precision": "fp64 (oracle)",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm


def stage_roofline(stage_ms, stage_n, prec, scheme, hbm_peak):
    out = []
    reals = 8 * NZ * NV
    for s in range(5):
        if stage_n[s] == 0:
            continue
        avg_ms = stage_ms[s] / stage_n[s]
        byts = STAGE_BYTES[prec][s] * reals
        gbs = byts / (avg_ms * 1e-3) / 1e9
        rec = {"kernel": KERNEL_NAMES[s], "stage": s + 1, "avg_ms": avg_ms, "alg_bytes": byts,
               "GB/s": gbs, "hbm_frac": gbs / hbm_peak, "total_ms": stage_ms[s]}
        winst = kernel_counts("warp_inst_per_cell") if prec == "mixed" else None
        if winst and f"{scheme}_{prec}" in winst and s < 4:
            # warp instructions per second against 4 per SM and clock (2.07 GHz)
            rate = winst[f"{scheme}_{prec}"][s] * 2 * NZ * NV / (avg_ms * 1e-3)
            rec["issue_frac"] = rate / (4 * SMS * 2.07e9)
        if prec == "fp64":
            fl = FP64_FLOPS_PER_CELL[scheme][s] * 2 * NZ * NV
            rec["fp64_tflops"] = fl / (avg_ms * 1e-3) / 1e12
            rec["fp64_alu_frac"] = rec["fp64_tflops"] / FP64_PEAK_TFLOPS
            ops = fp64_pipe_ops()
            if ops is not None:  # pipe lane-operations per second against the FMA rate
                rate = ops[scheme][s] * 2 * NZ * NV / (avg_ms * 1e-3)
                rec["fp64_pipe_frac"] = rate / (FP64_PEAK_TFLOPS * 1e12 / 2)
        out.append(rec)
    return out


def run_variant(b, scheme, prec, steps, warmup, device, stream, state_dev):
    import torch
    h = b.cosenu_create(NZ, NV, L, SCHEMES[scheme], PRECS[prec])
    try:
        b.cosenu_set_stream(h, stream.cuda_stream)
        b.cosenu_set_params(h, mu=MU)
        b.cosenu_set_state_device(h, state_dev.data_ptr(), state_dev.numel())
        b.cosenu_step(h, warmup)
        b.cosenu_sync(h)
        torch.cuda.synchronize(device)
        b.cosenu_set_stage_timing(h, True)
        b.cosenu_stage_times(h)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.cosenu_step(h, steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        sms, sn = b.cosenu_stage_times(h)
        b.cosenu_sync(h)
        return ms, sms, sn
    finally:
        b.cosenu_destroy(h)


# The two smaller configurations of the method's workloads (nz, nv, L, steps per
# timed run for mixed / FP64, legs).  The first is L2-resident and launch-bound:
# its steps replay a CUDA graph, reported as microseconds per step.
SMALL_CONFIGS = (
    ("nz=512, nv=32, z in [-50, 50), mu=1", 512, 32, 100.0, (400, 400),
     (("fdko", "fp64"), ("fdko", "mixed"), ("weno7", "fp64"), ("weno7", "mixed"))),
    ("nz=65536, nv=128, z in [-1600, 1600), mu=1", 65536, 128, 3200.0, (20, 4),
     (("fdko", "mixed"), ("weno7", "mixed"), ("fdko", "fp64"), ("weno7", "fp64"))),
)


def run_small_configs(b, device, stream):
    """Per-step time of the smaller configurations (alpha=0.9, sigma=(0.6, 0.5),
    random-phase seed 1e-6, dt = 0.4 dz), steps replayed from the handle's graph."""
    import torch

    from paper_2203_12866_gb300 import inputs
    out = {}
    for label, nz, nv, lz, (k_mixed, k_fp64), legs in SMALL_CONFIGS:
        with torch.cuda.stream(stream):
            st = inputs.collective_state_device(nz, nv, device, alpha=ALPHA, sigma_nu=SIG_NU,
                                                sigma_nubar=SIG_NUBAR, eps0=EPS0, seed=SEED)
        stream.synchronize()
        for sc, pr in legs:
            k = k_mixed if pr == "mixed" else k_fp64
            h = b.cosenu_create(nz, nv, lz, SCHEMES[sc], PRECS[pr])
            try:
                b.cosenu_set_stream(h, stream.cuda_stream)
                b.cosenu_set_params(h, mu=1.0)
                b.cosenu_set_state_device(h, st.data_ptr(), st.numel())
                b.cosenu_step(h, 4)
                b.cosenu_sync(h)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                b.cosenu_step(h, k)
                e1.record(stream)
                e1.synchronize()
                if b.cosenu_sync(h) != 0:
                    raise RuntimeError(f"{label} {sc} {pr}: solver error")
                ms = e0.elapsed_time(e1) / k
            finally:
                b.cosenu_destroy(h)
            out[f"{sc}_{pr}_{nz}x{nv}"] = {"workload": label, "scheme": sc, "precision": pr,
                                           "steps": k, "us_per_step": ms * 1e3,
                                           "cell_updates_per_s": 2 * nz * nv / (ms * 1e-3)}
        del st
    torch.cuda.empty_cache()
    return out


BATCH_WORKLOAD = ("batched run: 256 independent grids, nz log-uniform [1024, 32768], "
                  "nv in {32, 64, 128}, mu log-uniform [0.1, 10], alpha U[0.7, 1.2], "
                  "sigma_nu, sigma_nubar U[0.3, 0.8], scheme FD+KO or WENO7 at random, "
                  "dz = 0.2/mu, dt = 0.4 dz, mixed precision, seed 12866")


def run_batched(args, device, hbm_peak):
    """The batched solver on the 256-grid workload: tuned launch shapes, then
    args.batch_steps steps timed with CUDA events on the batch's stream."""
    import torch

    from paper_2203_12866_gb300 import binding as b
    from paper_2203_12866_gb300 import inputs

    specs = inputs.batch_instances(args.batch_n)
    bt = b.Batch()
    try:
        cells = reals = 0
        for sp in specs:
            m = bt.add(sp["nz"], sp["nv"], sp["L"], sp["scheme"], b.COSENU_MIXED, mu=sp["mu"],
                       dt=sp["dt"])
            st = inputs.collective_state_device(sp["nz"], sp["nv"], device, alpha=sp["alpha"],
                                                sigma_nu=sp["sigma_nu"],
                                                sigma_nubar=sp["sigma_nubar"], seed=sp["seed"])
            torch.cuda.synchronize(device)
            b.cosenu_set_state_device(m.h, st.data_ptr(), st.numel())
            torch.cuda.synchronize(device)
            del st
            cells += 2 * sp["nz"] * sp["nv"]
            reals += 8 * sp["nz"] * sp["nv"]
        t0 = time.perf_counter()
        tuned = bt.tune(reps=1)
        tune_s = time.perf_counter() - t0
        bt.step(args.warmup)
        rc, bad = bt.sync()
        stream = torch.cuda.ExternalStream(b.cosenu_batch_stream(bt.b), device=device)
        l0 = b.cosenu_kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.step(args.batch_steps)
        e1.record(stream)
        e1.synchronize()
        launches = b.cosenu_kernel_launches() - l0
        ms = e0.elapsed_time(e1) / args.batch_steps
        # per-kernel device times of a few directly launched steps (classes in series)
        b.cosenu_batch_set_stage_timing(bt.b, True)
        b.cosenu_batch_stage_times(bt.b)
        bt.step(2)
        kms, kn = b.cosenu_batch_stage_times(bt.b)
        b.cosenu_batch_set_stage_timing(bt.b, False)
        rc2, bad2 = bt.sync()
        alg = sum(STAGE_BYTES["mixed"]) * reals
        classes = bt.classes()
        for c in classes:  # achieved bandwidth of each class's kernels
            creals = 8 * c["rows"] * c["nv"]
            c["kernel_GBs"] = [STAGE_BYTES["mixed"][k] * creals / (ms_k * 1e-3) / 1e9
                               if ms_k > 0 else None for k, ms_k in enumerate(c["kernel_ms"])]
            c["class_ms_per_step"] = sum(c["kernel_ms"])
        return {
            "workload": BATCH_WORKLOAD, "grids": len(specs), "cells_per_step": cells,
            "value": cells / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms,
            "steps": args.batch_steps, "warmup": args.warmup, "tune_steps": tuned,
            "tune_s": tune_s, "gpu_launches": launches,
            "hbm": {"achieved": alg / (ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": alg / (ms * 1e-3) / 1e9 / hbm_peak,
                    "alg_bytes_per_step": alg, "bytes_per_real": sum(STAGE_BYTES["mixed"])},
            "kernel_ms_per_step": {KERNEL_NAMES[k]: float(kms[k] / 2) for k in range(5)},
            "classes": classes, "device_bytes": bt.device_bytes(),
            "flags": [rc, bad, rc2, bad2],
        }
    finally:
        bt.close()
        torch.cuda.empty_cache()


SERVE_WORKLOAD = ("serving trace: Poisson arrivals, grids from the batched-run recipe, precision "
                  "alternating mixed / FP64, t_final U[50, 500]/mu, 64 GB workspace budget")


def serve_trace(b, trace, budget, rate_scale=1.0, max_running=0, precision=None):
    """Submit the trace's runs at their arrival times (divided by rate_scale), wait for
    all, and summarise time-to-solution (submission to result, queueing included)."""
    srv = b.Server(budget, max_running=max_running)
    try:
        t0 = time.perf_counter()
        tickets = []
        for r in trace:
            delay = t0 + r["t_arrival"] / rate_scale - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            req = b.make_request(r["nz"], r["nv"], r["L"], r["scheme"],
                                 r["precision"] if precision is None else precision,
                                 nsteps=r["nsteps"], alpha=r["alpha"], sigma_nu=r["sigma_nu"],
                                 sigma_nubar=r["sigma_nubar"], eps0=1e-6, seed=r["seed"],
                                 mu=r["mu"], dt=r["dt"])
            tickets.append(srv.submit(req))
        res = [srv.wait(t, 3600.0)[1] for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    lat = sorted(r["t_done"] - r["t_submit"] for r in res)
    span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    cu = sum(2 * r["nz"] * r["nv"] * r["nsteps"] for r in trace)
    q = lambda p: float(np.percentile(lat, p))  # noqa: E731
    return {"requests": len(trace), "offered_rate_per_s": len(trace) / (trace[-1]["t_arrival"] /
                                                                         rate_scale),
            "p50_s": q(50), "p99_s": q(99), "mean_s": float(np.mean(lat)), "max_s": lat[-1],
            "makespan_s": span, "completed_per_s": len(trace) / span,
            "cell_updates_per_s": cu / span, "statuses": sorted({r["status"] for r in res}),
            "peak_workspace_bytes": st["peak_bytes"], "budget_bytes": st["budget"],
            "rounds": st["rounds"], "max_running": max_running}


def run_serving(args):
    """Continuous batching on the serving trace (at most --serve-max-running runs in the
    batch at once).  Leads with arrivals stretched to 70% of the capacity the loop
    measures on the trace's own burst of arrivals (50 per second: all runs queued
    almost at once, a throughput figure).  On the same 70% arrivals, the runs served one at a time, each at its
    own precision (the same accuracy), and all in FP64 (the plain single-instance
    path); and the burst served one at a time at each run's own precision (the
    throughput comparison under overload)."""
    from paper_2203_12866_gb300 import binding as b
    from paper_2203_12866_gb300 import inputs

    trace = inputs.serving_trace(args.serve_requests, args.serve_rate,
                                 step_scale=args.serve_step_scale)
    budget = 64 << 30
    mr = args.serve_max_running
    burst = serve_trace(b, trace, budget, max_running=mr)  # the capacity measurement
    cap = burst["completed_per_s"]
    scale = 0.7 * cap / args.serve_rate  # arrival times stretched to 70% of capacity
    out = {"workload": SERVE_WORKLOAD, "rate_per_s": args.serve_rate,
           "step_scale": args.serve_step_scale,
           "steps_range": [min(r["nsteps"] for r in trace), max(r["nsteps"] for r in trace)],
           "cell_updates": sum(2 * r["nz"] * r["nv"] * r["nsteps"] for r in trace)}
    out["batched_70pct"] = serve_trace(b, trace, budget, rate_scale=scale, max_running=mr)
    out["batched_burst"] = burst
    if args.serve_baselines:
        out["one_at_a_time_70pct"] = serve_trace(b, trace, budget, rate_scale=scale,
                                                 max_running=1)
        out["fp64_one_at_a_time_70pct"] = serve_trace(b, trace, budget, rate_scale=scale,
                                                      max_running=1, precision=b.COSENU_FP64)
        out["one_at_a_time_burst"] = serve_trace(b, trace, budget, max_running=1)
    return out


def summary(value, ms_step, roofline, variants, small, batched, serving):
    """The line's key figures in a few hundred characters, placed last."""
    r3 = lambda x: None if x is None else float(f"{x:.4g}")  # noqa: E731
    out = {"ms_per_step": r3(ms_step), "value": r3(value), "step_hbm_frac": r3(roofline["step_frac"]),
           "dominant_frac": r3(roofline["frac"])}
    if variants:
        out["variants_ms_per_step"] = {k: r3(v["ms_per_step"]) for k, v in variants.items()}
        out["fp64_pipe_frac"] = {k: r3(v["fp64_pipe_frac"]) for k, v in variants.items()
                                 if "fp64_pipe_frac" in v}
        out["issue_frac"] = {k: [r3(st["issue_frac"]) for st in v["stages"] if "issue_frac" in st]
                             for k, v in variants.items()
                             if any("issue_frac" in st for st in v["stages"])}
    if small:
        out["small_us_per_step"] = {k: r3(v["us_per_step"]) for k, v in small.items()}
    if batched:
        out["batched"] = {"ms_per_step": r3(batched["ms_per_step"]), "value": r3(batched["value"]),
                          "hbm_frac": r3(batched["hbm"]["frac"]),
                          "launches_per_step": r3(batched["gpu_launches"] / batched["steps"])}
    if serving:
        out["serving_p50_p99_s"] = {k: [r3(v["p50_s"]), r3(v["p99_s"])] for k, v in serving.items()
                                    if isinstance(v, dict) and "p50_s" in v}
    return out


def run_ours(args, world, rank, local):
    import torch

    from paper_2203_12866_gb300 import binding as b
    from paper_2203_12866_gb300 import inputs

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    b.load()
    hbm_peak, peak_kind = peaks()
    stream = torch.cuda.Stream(device)
    scheme, prec = args.scheme, args.precision
    cells = 2 * NZ * NV

    # ---- main timed region: inputs resident in HBM
    h = b.cosenu_create(NZ, NV, L, SCHEMES[scheme], PRECS[prec])
    b.cosenu_set_stream(h, stream.cuda_stream)
    b.cosenu_set_params(h, mu=MU)
    with torch.cuda.stream(stream):
        state = inputs.collective_state_device(NZ, NV, device, alpha=ALPHA, sigma_nu=SIG_NU,
                                               sigma_nubar=SIG_NUBAR, eps0=EPS0, seed=SEED)
    stream.synchronize()
    b.cosenu_set_state_device(h, state.data_ptr(), state.numel())
    b.cosenu_step(h, args.warmup)
    b.cosenu_sync(h)
    b.cosenu_set_stage_timing(h, True)
    b.cosenu_stage_times(h)
    torch.cuda.synchronize(device)
    barrier(world, device)
    torch.cuda.synchronize(device)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = b.cosenu_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.cosenu_step(h, args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize(device)
    launches = b.cosenu_kernel_launches() - l0
    barrier(world, device)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stage_ms, stage_n = b.cosenu_stage_times(h)
    b.cosenu_sync(h)
    cons = b.cosenu_conserved(h)
    ms_max = dist_max(ms, world, device)
    ms_step = ms_max / args.steps
    value = world * cells / (ms_step * 1e-3)
    stages = stage_roofline(stage_ms, stage_n, prec, scheme, hbm_peak)
    dom = max(stages, key=lambda r: r["total_ms"])
    traffic = ncu_traffic(scheme, prec, dom["stage"])
    roofline = {"bound": "hbm", "achieved": dom["GB/s"], "peak": hbm_peak, "unit": "GB/s",
                "frac": dom["hbm_frac"], "traffic": traffic,
                "kernel": (f"rk4_stage_kernel<{scheme},{prec},stage {dom['stage']}>"
                           if dom["stage"] <= 4 else "apply_increment_kernel"),
                "peak_kind": f"{peak_kind} (copy)", "frac_of_nominal": dom["GB/s"] / NOMINAL_HBM_GBS,
                "stages": stages,
                "step_frac": (sum(STAGE_BYTES[prec]) * 8 * NZ * NV / (ms_step * 1e-3) / 1e9)
                / hbm_peak}

    # ---- end to end through the C ABI with host buffers: each step copies the
    # state in from pinned host memory, steps, and reads the new state back
    e2e = None
    if args.e2e_steps > 0:
        n = 8 * NZ * NV
        host = torch.empty(n, dtype=torch.float64, pin_memory=True)
        hp = host.numpy()
        b.cosenu_get_state(h, hp)
        b.cosenu_set_state(h, hp)  # warm the path
        b.cosenu_step(h, 1)
        b.cosenu_get_state(h, hp)
        barrier(world, device)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            b.cosenu_set_state(h, hp)
            b.cosenu_step(h, 1)
            b.cosenu_get_state(h, hp)
        sec = dist_max(time.perf_counter() - t0, world, device)
        e2e = {"value": world * cells * args.e2e_steps / sec, "unit": "cell-updates/s",
               "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8,
               "steps": args.e2e_steps, "api": "cosenu_set_state + cosenu_step(1) + cosenu_get_state"}
        del host, hp
    b.cosenu_destroy(h)

    # ---- the other (scheme, precision) variants on the same input
    variants = {}
    if args.variants:
        for sc in ("fdko", "weno7"):
            for pr in ("mixed", "fp64"):
                if (sc, pr) == (scheme, prec):
                    continue
                k = args.variant_steps if pr == "mixed" else max(1, args.variant_steps // 4)
                vms, vsm, vsn = run_variant(b, sc, pr, k, 1, device, stream, state)
                vst = stage_roofline(vsm, vsn, pr, sc, hbm_peak)
                rec = {"value": cells / (vms / k * 1e-3), "ms_per_step": vms / k, "steps": k,
                       "step_hbm_frac": (sum(STAGE_BYTES[pr]) * 8 * NZ * NV /
                                         (vms / k * 1e-3) / 1e9) / hbm_peak,
                       "stages": vst}
                if pr == "fp64":
                    fl = sum(FP64_FLOPS_PER_CELL[sc]) * cells
                    rec["bound"] = "alu"
                    rec["fp64_tflops"] = fl / (vms / k * 1e-3) / 1e12
                    rec["fp64_alu_frac"] = rec["fp64_tflops"] / FP64_PEAK_TFLOPS
                    ops = fp64_pipe_ops()
                    if ops is not None:  # the whole step against the FP64 pipe's rate
                        rate = sum(ops[sc]) * cells / (vms / k * 1e-3)
                        rec["fp64_pipe_frac"] = rate / (FP64_PEAK_TFLOPS * 1e12 / 2)
                    rec["fp64_peak_tflops"] = FP64_PEAK_TFLOPS
                    rec["fp64_peak_kind"] = FP64_PEAK_KIND
                variants[f"{sc}_{pr}"] = rec
    del state
    torch.cuda.empty_cache()

    small = run_small_configs(b, device, stream) if args.variants else None
    batched = run_batched(args, device, hbm_peak) if args.batched else None
    serving = run_serving(args) if args.serving and rank == 0 else None

    # ---- oracle on the host cores (rank 0, one GPU only)
    cpu = None
    if args.cpu_baseline and world == 1 and rank == 0:
        rate, sec, thr = oracle_rate(args.cpu_rows, args.cpu_steps, scheme)
        cpu = {"value": rate, "unit": "cell-updates/s", "cores": thr, "kind": "oracle",
               "sample": f"z-slab of {args.cpu_rows} rows x nv=256 x 2 species, {args.cpu_steps} "
                         f"RK4 steps ({sec:.1f} s), FP64 {scheme}, same dz and parameters"}

    if rank == 0:
        line = {
            "metric": "cell-updates/s (z*v*species per RK4 step)", "value": value,
            "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if NZ == NZ_FULL else f"PROFILING SIZE nz={NZ}",
                       "scheme": "FD+KO" if scheme == "fdko" else "WENO7",
                       "precision": prec, "nz": NZ, "nv": NV, "cells_per_step": cells,
                       "l2": "inputs larger than L2 (state 17.2 GB >> 129 MB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "variants": variants, "small_configs": small, "batched": batched,
            "serving": serving,
            "conserved_after": {"tr_nu": cons["tr_nu"], "M": list(cons["M"]),
                                "dP_max": cons["dP_max"]},
            "summary": summary(value, ms_step, roofline, variants, small, batched, serving),
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scheme", default="fdko", choices=["fdko", "weno7"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--variant-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-rows", type=int, default=65536)
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--batch-n", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--no-serving", dest="serving", action="store_false")
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-step-scale", type=float, default=0.1,
                    help="fraction of each run's t_final simulated (1 = the full trace)")
    ap.add_argument("--no-serve-baselines", dest="serve_baselines", action="store_false",
                    help="skip the one-at-a-time legs")
    ap.add_argument("--serve-max-running", type=int, default=8,
                    help="most runs batched at once in the continuous-batching legs (0: no limit)")
    ap.add_argument("--nz", type=int, default=NZ_FULL,
                    help="z cells (smaller values only for profiling captures)")
    args = ap.parse_args()
    global NZ, L
    NZ, L = args.nz, args.nz * DZ
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
