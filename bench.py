"""Benchmark of the GB300 compact gas-kinetic scheme (one JSON line on rank 0).

Headline workload: 2D Euler isentropic vortex (strength 5, gamma 1.4) on periodic [0,10]^2,
2048^2 cells, 8th-order compact linear reconstruction, fixed dt = CFL 0.3.  A step is one
full two-stage MSMD step (both face sweeps and both updates, twice).  Both forms run on the
same input: the FP32-bulk form (the headline value) and the plain FP64 form; each reports its
L1 density error against the exact (translated) solution at the end of its run.  Each form
is timed twice over the same number of steps: as the CUDA-graph replay that gks_steps runs
(the value) and as plain launches between per-launch CUDA events (gks_steps_timed: the
per-kernel times and the roofline of the longest launch).
Metric: cell-updates/s = cells * steps / seconds (whole job: summed over ranks).

The default line also carries two sub-objects measured in the same run: "shear", the 4096^2
Navier-Stokes double shear layer (8th-order WENO-Z, both forms), and "batch", 512 mixed
independent problems in one persistent launch per step (FP32-bulk, autotuned tiles).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gks|reference] [--n 2048]
                  [--workload vortex|shear|batch] [--no-sub]

--impl reference times the FP64 CPU oracle (the plain implementation the tests check the
GPU against) on the host cores, on bounded windows of the same workload.
Under torchrun each rank runs an independent replica of the workload (the problems do not
exchange data): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell-updates/s (2D 8th-order GKS, FP32-bulk vs FP64, isentropic vortex)"
METRIC_SHEAR = "cell-updates/s (2D 8th-order GKS, FP32-bulk vs FP64, Navier-Stokes WENO-Z shear layer)"


def metric_of(args):
    return METRIC_SHEAR if args.workload == "shear" else METRIC
UNIT = "cell-updates/s"
CFL = 0.3
# Per-unit figures of the kernels of a step (2D, 8th order, linear Euler).  unit: "face"
# (sweeps) or "cell" (updates).  f32 / f64: floating-point operations per unit (FMA = 2) from
# ncu's executed-instruction counters (FP32-bulk form: a 1024^2 capture; FP64 form: 256^2);
# bytes: algorithmic bytes per unit (each datum read or written once), given for the updates,
# whose limit is memory or the FP64 pipe (the sweeps are compute-side: issue-bound, DRAM below
# 20 %); traffic: DRAM bytes (read + write) per unit of a full-size launch (2048^2, one-pass
# dram__bytes capture of the benchmark's own step), scaled by the units a launch processes.
# The FP64 form has no traffic figure: its 256^2 capture fits in L2.  winstr: executed
# warp-instructions per 32 units (same captures), for the instruction-issue rate the sweeps
# are limited by (reported beside the roofline).
KERNEL_MODEL = {
    ("linear_euler", "fp64", "x_faces_stage1"): {"unit": "face", "f64": 1961.2, "winstr": 7353},
    ("linear_euler", "fp64", "y_faces_stage1"): {"unit": "face", "f64": 1809.6, "winstr": 5962},
    ("linear_euler", "fp64", "x_faces_stage2"): {"unit": "face", "f64": 1826.2, "winstr": 6914},
    ("linear_euler", "fp64", "y_faces_stage2"): {"unit": "face", "f64": 1674.6, "winstr": 5570},
    ("linear_euler", "fp32", "x_faces_stage1"): {"unit": "face", "f32": 2129.1, "f64": 35.0, "traffic": 180.8,
                                                 "winstr": 2092},
    ("linear_euler", "fp32", "y_faces_stage1"): {"unit": "face", "f32": 2052.5, "f64": 35.0, "traffic": 179.0,
                                                 "winstr": 1941},
    ("linear_euler", "fp32", "update_stage1"): {"unit": "cell", "f32": 84.0, "f64": 0.0, "bytes": 224.0,
                                                "traffic": 213.6, "winstr": 251},
    ("linear_euler", "fp32", "x_faces_stage2"): {"unit": "face", "f32": 1824.6, "f64": 4.0, "traffic": 134.4,
                                                 "winstr": 1626},
    ("linear_euler", "fp32", "y_faces_stage2"): {"unit": "face", "f32": 1747.0, "f64": 4.0, "traffic": 133.3,
                                                 "winstr": 1483},
    ("linear_euler", "fp32", "update_stage2"): {"unit": "cell", "f32": 44.0, "f64": 24.0, "bytes": 320.0,
                                                "traffic": 309.2, "winstr": 608},
    # 8th-order WENO-Z Navier-Stokes sweeps (double shear layer), FP32-bulk form: executed
    # FFMA x 2 + FMUL + FADD (and DFMA x 2 + DMUL + DADD) per face and warp-instructions per
    # 32 faces from one-pass instruction-counter captures of the 4096^2 step (the FP64 count
    # depends on the grid through dt/tau: the time coefficients' series length follows it)
    ("wenoz_ns", "fp32", "x_faces_stage1"): {"unit": "face", "f32": 10605.3, "f64": 238.3, "winstr": 9619},
    ("wenoz_ns", "fp32", "y_faces_stage1"): {"unit": "face", "f32": 10168.9, "f64": 238.3, "winstr": 9168},
    ("wenoz_ns", "fp32", "x_faces_stage2"): {"unit": "face", "f32": 10041.3, "f64": 141.3, "winstr": 8601},
    ("wenoz_ns", "fp32", "y_faces_stage2"): {"unit": "face", "f32": 9604.9, "f64": 141.3, "winstr": 8192},
    ("wenoz_ns", "fp32", "update_stage1"): {"unit": "cell", "f32": 84.0, "f64": 0.0, "bytes": 224.0},
    ("wenoz_ns", "fp32", "update_stage2"): {"unit": "cell", "f32": 44.0, "f64": 24.0, "bytes": 320.0},
}
HBM_FALLBACK_GBS = 6800.0


def hbm_peak():
    """HBM copy bandwidth in GB/s and its source: the measured copy bandwidth of this machine
    (MEASURED_PEAKS.json) when present."""
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError, TypeError):
        return HBM_FALLBACK_GBS, "of fallback (6.8 TB/s GB300 copy bandwidth)"


def roofline(form, name, ms, nx, ny, order, peak64, peak32, issue_peak=None, path="linear_euler"):
    """Roofline of one launch of kernel `name` taking `ms` milliseconds: the fraction of the
    FP32 and FP64 peaks (probes measured in this run) and of the HBM bandwidth, the largest
    named as the bound, the others listed beside it.  With issue_peak (warp-instructions per
    second the SMs can issue), the launch's instruction-issue rate is listed beside them too
    (executed instructions are not algorithmic work, so it is never the headline bound)."""
    m = KERNEL_MODEL.get((path, form, name)) if order == 8 else None
    if m is None:
        return {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "kernel": name}
    if m["unit"] == "face":
        units = (nx + 1) * ny if name.startswith("x") else nx * (ny + 1)
    else:
        units = nx * ny
    sec = ms * 1e-3
    cands = []
    if m.get("f32"):
        a = m["f32"] * units / sec
        cands.append({"bound": "alu", "achieved": a / 1e12, "peak": peak32 / 1e12, "unit": "TFLOP/s",
                      "frac": a / peak32, "peak_source": "FP32 FMA-chain probe measured in this run",
                      "pipe": "fp32", "flops_per_" + m["unit"]: m["f32"]})
    if m.get("f64"):
        a = m["f64"] * units / sec
        cands.append({"bound": "alu", "achieved": a / 1e12, "peak": peak64 / 1e12, "unit": "TFLOP/s",
                      "frac": a / peak64, "peak_source": "FP64 FMA-chain probe measured in this run",
                      "pipe": "fp64", "flops_per_" + m["unit"]: m["f64"]})
    if m.get("bytes"):
        hpeak, hsrc = hbm_peak()
        a = m["bytes"] * units / sec / 1e9
        cands.append({"bound": "hbm", "achieved": a, "peak": hpeak, "unit": "GB/s", "frac": a / hpeak,
                      "peak_source": hsrc, "bytes_per_" + m["unit"]: m["bytes"]})
    cands.sort(key=lambda c: -c["frac"])
    main = dict(cands[0])
    main["kernel"] = name
    main["traffic"] = m["traffic"] * units if m.get("traffic") else None
    main["other_bounds"] = [{k: c[k] for k in ("bound", "achieved", "peak", "unit", "frac")} for c in cands[1:]]
    if issue_peak and m.get("winstr"):
        a = m["winstr"] / 32.0 * units / sec
        main["other_bounds"].append({"bound": "issue", "achieved": a / 1e9, "peak": issue_peak / 1e9,
                                     "unit": "G warp-instructions/s", "frac": a / issue_peak,
                                     "peak_source": "4 per clock per SM x SMs x median SM clock under load"})
    return main


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gks", choices=["gks", "reference"])
    ap.add_argument("--n", type=int, default=None,
                    help="grid side (default 2048 for vortex, 4096 for shear)")
    ap.add_argument("--order", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-acc", action="store_true", help="skip the L1 error against the exact solution")
    ap.add_argument("--precision", default="both", choices=["both", "fp32", "fp64"])
    ap.add_argument("--workload", default="vortex", choices=["vortex", "shear", "batch"],
                    help="vortex: the 2D benchmark workload (8th-order linear isentropic vortex); "
                         "shear: the Navier-Stokes double shear layer (8th-order WENO-Z, 4096^2); "
                         "batch: the mixed batch of 512 problems (persistent launch, FP32-bulk)")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--no-sub", action="store_true",
                    help="headline workload only (no shear / batch sub-objects in the line)")
    ap.add_argument("--shear-n", type=int, default=4096)
    ap.add_argument("--shear-steps", type=int, default=9,
                    help="timed steps of the shear sub-object (FP32-bulk; the FP64 form a third)")
    ap.add_argument("--batch-steps", type=int, default=20)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# Replica timing over ranks (one process per GPU, each advancing its own problems; no data
# exchange between ranks): the job's time is the slowest rank's, its work the sum of all
# ranks' work.  dist is torch.distributed (or None for one process); device holds the
# reduction tensor ("cuda" under NCCL, "cpu" under gloo).
def reduce_over_ranks(value, dist, device, op="max"):
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_per_rank, ms_per_rank, steps, dist, device):
    """Units per second of the whole job: all ranks' units over the slowest rank's time."""
    units = reduce_over_ranks(units_per_rank, dist, device, "sum")
    ms = reduce_over_ranks(ms_per_rank, dist, device, "max")
    return units * steps / (ms * 1e-3), ms


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def pinned_copy_gbs(n, reps=5):
    """Host link bandwidth for one state: n float64 values copied between pinned host memory
    and the device, each direction timed alone with CUDA events (the floor of the e2e step)."""
    import torch
    h = torch.empty(n, dtype=torch.float64).pin_memory()
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    d.copy_(h, non_blocking=True)
    h.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    out = {}
    for name, dst, src in (("h2d", d, h), ("d2h", h, d)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            dst.copy_(src, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        out[name] = reps * n * 8 / (a.elapsed_time(b) * 1e-3) / 1e9
    del h, d
    return out


def window_state(st, w):
    """The w x w window at the centre of the workload (through the vortex core, or across a
    shear layer), as a problem of its own with transmissive edges."""
    w = min(w, st.nx, st.ny)
    i0, j0 = (st.nx - w) // 2, (st.ny - w) // 2
    sl = (slice(None), slice(j0, j0 + w), slice(i0, i0 + w))
    from paper_1901_00261_gb300 import inputs
    return inputs.State(np.ascontiguousarray(st.W[sl]), np.ascontiguousarray(st.Wx[sl]),
                        np.ascontiguousarray(st.Wy[sl]), w, w, st.gamma, 0.0, w * st.dx, 0.0,
                        w * st.dy, 1, 1, mu=st.mu, Pr=st.Pr, order=st.order, recon=st.recon)


def cpu_baseline(st, dt, budget_s=12.0, window=128, keep=None):
    """The oracle as it stands, on the host cores, on a window of the same workload
    (transmissive window edges), as many steps as fit in the time budget.  keep (a dict):
    receives the window problem, the step count and the oracle's final state."""
    import oracle
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    ws = window_state(st, window)
    w = ws.nx
    O = oracle.Solver(w, w, ws.gamma, ws.mu, ws.Pr, ws.order, ws.recon, 1, 1, ws.x0, ws.x1, ws.y0, ws.y1)
    O.set_state(ws.W, ws.Wx, ws.Wy)
    t0 = time.perf_counter()
    steps = 0
    while True:
        O.step(dt)
        steps += 1
        el = time.perf_counter() - t0
        if el > budget_s or steps >= 50:
            break
    value = w * w * steps / el
    if keep is not None:
        keep.update(window=ws, steps=steps, state=O.get_state())
    return {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"{w}x{w} window at the centre of the {st.nx}x{st.ny} workload, {steps} steps, {el:.1f} s"}


def cpu_single_thread(st, dt, budget_s=4.0, window=64):
    """The oracle on one host thread, on a smaller window of the same workload (the
    per-core rate beside the all-core cpu_baseline)."""
    import oracle
    threads = oracle.get_threads()
    oracle.set_threads(1)
    try:
        ws = window_state(st, window)
        O = oracle.Solver(ws.nx, ws.ny, ws.gamma, ws.mu, ws.Pr, ws.order, ws.recon, 1, 1,
                          ws.x0, ws.x1, ws.y0, ws.y1)
        O.set_state(ws.W, ws.Wx, ws.Wy)
        t0 = time.perf_counter()
        steps = 0
        while True:
            O.step(dt)
            steps += 1
            el = time.perf_counter() - t0
            if el > budget_s or steps >= 50:
                break
    finally:
        oracle.set_threads(threads)
    return {"value": ws.nx * ws.ny * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{ws.nx}x{ws.ny} window at the centre, {steps} steps, {el:.1f} s"}


def vs_oracle(keep, dt, forms):
    """Both GPU forms on the oracle's window problem, same dt and step count: the L1 density
    difference and the largest per-variable difference relative to max |W| (cell averages)."""
    from paper_1901_00261_gb300 import gks
    ws, steps, (Wo, _, _) = keep["window"], keep["steps"], keep["state"]
    out = {"window": f"{ws.nx}x{ws.ny} centre, transmissive edges", "steps": steps}
    for form in forms:
        prec = gks.PREC_FP32_BULK if form == "fp32" else gks.PREC_FP64
        G = gks.Solver.from_state(ws, precision=prec)
        G.steps(dt, steps)
        W = G.get_state()[0]
        G.close()
        out[form] = {"l1_rho": float(np.abs(W[0] - Wo[0]).mean()),
                     "linf_rel": float(max(np.abs(W[v] - Wo[v]).max() / np.abs(Wo[v]).max()
                                           for v in range(W.shape[0])))}
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_1901_00261_gb300 import inputs
    if args.workload == "shear":
        st = inputs.shear_layer_2d(args.n, order=args.order)
    else:
        st = inputs.isentropic_vortex_2d(args.n, order=args.order, recon=0)
    import oracle
    O = oracle.Solver(8, 8)  # builds the library before timing
    del O
    # dt of the full workload
    rho = st.W[0]
    U, V = st.W[1] / rho, st.W[2] / rho
    p = 0.4 * (st.W[3] - 0.5 * rho * (U * U + V * V))
    c = np.sqrt(1.4 * p / rho)
    dt = CFL / ((np.abs(U) + c) / st.dx + (np.abs(V) + c) / st.dy).max()
    # each step is a bounded sample (about two minutes for the whole run)
    budget = max(0.5, min(8.0, 120.0 / max(1, args.steps)))
    per_step = []
    for _ in range(args.warmup):
        cpu_baseline(st, dt, budget_s=min(2.0, budget), window=64)
    for _ in range(args.steps):
        per_step.append(cpu_baseline(st, dt, budget_s=budget, window=96))
    val = statistics.median([r["value"] for r in per_step])
    cb = dict(per_step[-1])
    cb["value"] = val
    line = {"impl": "reference", "metric": metric_of(args), "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * st.nx * st.ny / val,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args):
    if args.workload == "shear":
        return {"workload": f"shear_layer_2d_ns_{args.n}x{args.n}", "cells": args.n * args.n,
                "order": args.order, "recon": "wenoz", "mu": 1e-4, "Pr": 0.72,
                "precision": "fp32-bulk (headline) and fp64", "cfl": CFL, "domain": "periodic [0,1]^2",
                "l2_policy": "inputs exceed L2 (state 12 x 8 B per cell)",
                "parallelism": f"replicas x{args.gpus}"}
    return {"workload": f"isentropic_vortex_2d_{args.n}x{args.n}", "cells": args.n * args.n,
            "order": args.order, "recon": "linear", "precision": "fp32-bulk (headline) and fp64", "cfl": CFL,
            "domain": "periodic [0,10]^2", "l2_policy": "inputs exceed L2 (state 12 x 8 B per cell)",
            "parallelism": f"replicas x{args.gpus}"}


def _build_spec(spec):
    from paper_1901_00261_gb300 import inputs
    return inputs.build_problem(spec)


def batch_measure(args, ws, rank, local, dist, steps):
    """Mixed batch: 1D Riemann problems (N log-uniform in [100, 20000], WENO-Z) and 2D
    vortices (side log-uniform in [64, 1024], linear), orders 6/8 from the seed; one
    persistent launch per step, tile shape chosen by the autotuner.  Returns the measured
    record (value, ms per step, clocks, configuration and autotuner table).

    Some of the random Riemann problems turn non-physical under the scheme within a few steps
    (no limiter; the same happens in the oracle).  The workload is first run untimed for the
    warm-up + timed step count; problems flagged there are dropped (listed in the record)
    and the batch is rebuilt from the rest, so that every timed cell-update is a real one."""
    import multiprocessing as mp
    from paper_1901_00261_gb300 import inputs
    specs = inputs.batch_specs(args.batch_count, seed=rank)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        states = pool.map(_build_spec, specs, chunksize=4)
    import torch
    from paper_1901_00261_gb300 import gks
    stream = torch.cuda.Stream()     # the batch runs on this stream; the events are recorded on it
    B = gks.Batch(states, stream=stream.cuda_stream)
    dts = CFL / B.max_wavespeed()
    B.steps(dts, args.warmup + steps)
    bad = [int(i) for i in np.nonzero(B.problem_status() != gks.GKS_OK)[0]]
    B.close()
    keep = [i for i in range(len(states)) if i not in set(bad)]
    states = [states[i] for i in keep]
    dts = dts[keep]
    B = gks.Batch(states, stream=stream.cuda_stream)
    report = B.autotune(dts, steps=2)
    B.steps(dts, args.warmup)
    B.sync()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    with ClockSampler(local) as clk:
        t0.record(stream)
        B.steps(dts, steps)
        t1.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    B.sync()      # raises if any kept problem failed inside the timed region
    cells = sum(st.nx * st.ny for st in states)
    value, ms = job_throughput(cells, t0.elapsed_time(t1), steps, dist, "cuda")
    fpt, bps = B.config()
    B.close()
    return {"metric": "cell-updates/s (batched mixed problems, FP32-bulk, persistent launch)",
            "value": value, "unit": UNIT, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms / steps,
            "dtype": "f32-bulk (f64 time coefficients and accumulation)",
            "config": {"workload": f"batch_{args.batch_count}_mixed", "problems": len(states),
                       "cells": cells,
                       "problems_1d": sum(1 for st in states if st.ny == 1),
                       "problems_2d": sum(1 for st in states if st.ny > 1),
                       "dropped_nonphysical": [dict(index=i, n=specs[i].n, order=specs[i].order,
                                                    left=specs[i].left, right=specs[i].right)
                                               for i in bad],
                       "faces_per_thread": fpt, "blocks_per_sm": bps,
                       "l2": "inputs larger than L2"},
            "gpu_launches": steps, "clocks": clk.summary(),
            "autotune": report.strip().splitlines()}


def run_batch(args, ws, rank, local):
    """--workload batch: the batch record as the JSON line of its own."""
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    r = batch_measure(args, ws, rank, local, dist, args.steps)
    if rank == 0:
        line = dict(r)
        line.update({"n_gpus": ws, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                     "data": "synthetic"})
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def measure_form(st, form, steps, warmup, stream, local, dist, peaks, path, order, want_acc):
    """One form of one solver workload: graph-replayed steps (the value), then the same number
    of plain-launch steps between per-launch CUDA events (per-kernel times, roofline)."""
    import torch
    from paper_1901_00261_gb300 import gks, inputs
    prec = gks.PREC_FP32_BULK if form == "fp32" else gks.PREC_FP64
    ncell = st.nx * st.ny
    G = gks.Solver.from_state(st, stream=stream.cuda_stream, precision=prec)
    dt = CFL / G.max_wavespeed()
    nl = G.launches_per_step()
    G.steps(dt, warmup)
    G.sync()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        G.steps(dt, steps)               # the captured two-stage step, replayed
        ev[1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    G.sync()
    value, ms = job_throughput(ncell, ev[0].elapsed_time(ev[1]), steps, dist, "cuda")
    with ClockSampler(local) as clk2:
        ev[2].record(stream)
        kernel_ms = G.steps_timed(dt, steps)
        ev[3].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    G.sync()
    value_plain, ms_plain = job_throughput(ncell, ev[2].elapsed_time(ev[3]), steps, dist, "cuda")
    per_launch = kernel_ms / steps
    slot_names = ["x_faces_stage1", "y_faces_stage1", "update_stage1",
                  "x_faces_stage2", "y_faces_stage2", "update_stage2"]
    k_dom = int(np.argmax(per_launch))
    csum = clk.summary()
    issue_peak = None
    try:
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        mhz = clk2.summary().get("sm_mhz") or csum.get("sm_mhz") or 2070.0
        issue_peak = 4.0 * sms * mhz * 1e6
    except Exception:
        issue_peak = None
    roof = roofline(form, slot_names[k_dom], float(per_launch[k_dom]), st.nx, st.ny, order,
                    peaks["fp64"], peaks["fp32"], issue_peak, path=path)
    r = {"value": value, "ms_per_step": ms / steps, "steps": steps, "gpu_launches": nl * steps,
         "api": "gks_steps (CUDA graph of the two-stage step, replayed)",
         "plain_launches": {"value": value_plain, "ms_per_step": ms_plain / steps,
                            "api": "gks_steps_timed (plain launches, CUDA events around each)",
                            "clocks": clk2.summary()},
         "roofline": roof, "clocks": csum,
         "kernel_ms_per_launch": {n: float(v) for n, v in zip(slot_names, per_launch)}}
    T = dt * (warmup + 2 * steps)
    r["t_end"] = T
    W = None
    if want_acc:
        W, _, _ = G.get_state()
        if path == "linear_euler":
            ex = inputs.vortex_exact_avg(st.nx, T)
            r["l1_rho_vs_exact"] = float(np.abs(W[0] - ex[0]).mean())
            r["linf_rho_vs_exact"] = float(np.abs(W[0] - ex[0]).max())
        W = W[0]
    return r, G, dt, W


def solver_workload(st, forms, steps, warmup, stream, local, dist, peaks, path, order, rank, no_acc):
    """Both forms of a single-grid workload; returns {form: record}, the L1 density difference
    of the two forms at the end, and the solver/dt of the first form."""
    out, Ws, keep = {}, {}, None
    for k, form in enumerate(forms):
        r, G, dt, W = measure_form(st, form, steps[form], warmup, stream, local, dist, peaks, path,
                                   order, want_acc=(not no_acc and rank == 0))
        out[form] = r
        if W is not None:
            Ws[form] = W
        if k == 0:
            keep = (G, dt)
        else:
            G.close()
    diff = None
    if len(Ws) == 2 and out["fp32"]["t_end"] == out["fp64"]["t_end"]:
        diff = float(np.abs(Ws["fp32"] - Ws["fp64"]).mean())
    return out, diff, keep


def main():
    args = parse()
    if args.n is None:
        args.n = 4096 if args.workload == "shear" else 2048
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "batch":
        run_batch(args, ws, rank, local)
        return
    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    from paper_1901_00261_gb300 import gks, inputs

    shear = args.workload == "shear"
    if shear:
        st = inputs.shear_layer_2d(args.n, order=args.order)
    else:
        st = inputs.isentropic_vortex_2d(args.n, order=args.order, recon=0)
    path = "wenoz_ns" if shear else "linear_euler"
    # the solvers run on this stream and the CUDA events are recorded on it (the legacy
    # default stream would leave the library to create a stream of its own)
    stream = torch.cuda.Stream()
    ncell = st.nx * st.ny

    peaks = {"fp64": gks.probe_alu_peak(True), "fp32": gks.probe_alu_peak(False)}
    forms = {"both": ["fp32", "fp64"], "fp32": ["fp32"], "fp64": ["fp64"]}[args.precision]
    steps = {"fp32": args.steps, "fp64": args.steps if not shear else max(1, args.steps // 4)}
    results, diff, (G, dt) = solver_workload(st, forms, steps, args.warmup, stream, local, dist, peaks,
                                             path, args.order, rank, args.no_acc)
    head = forms[0]
    # end to end through the public API with host buffers: per step, H2D of the state from
    # pinned memory, one step, D2H of the resulting state into pinned memory.  Headline: the
    # pipelined call (gks_step_host_async: copy-in, step and copy-out of consecutive steps
    # overlap); beside it the same work as set_state + step + get_state, one after another.
    e2e = None
    if not args.no_e2e:
        e_steps = min(args.steps, 50)
        Wp = torch.from_numpy(st.W).pin_memory().numpy()
        Wxp = torch.from_numpy(st.Wx).pin_memory().numpy()
        Wyp = torch.from_numpy(st.Wy).pin_memory().numpy()
        ins = (Wp, Wxp, Wyp)
        outs = [[torch.empty(st.W.shape, dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
                for _ in range(3)]
        for k in range(3):
            G.step_host_async(ins, outs[k], dt)
        G.sync()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        # three runs of e_steps calls; the median run is the value (the runtime places the two
        # copy directions on the copy engines per run, and in some runs they do not overlap)
        runs = []
        for _ in range(3):
            tw = time.perf_counter()
            for k in range(e_steps):
                G.step_host_async(ins, outs[k % 3], dt)
            G.sync()
            runs.append(time.perf_counter() - tw)
        el = statistics.median(runs)
        L = gks.lib()
        ptr = lambda a: a.ctypes.data_as(gks.ctypes.c_void_p)  # noqa: E731
        o = outs[0]
        torch.cuda.synchronize()
        ts = time.perf_counter()
        for _ in range(e_steps):
            G.set_state(Wp, Wxp, Wyp)
            G.step(dt)
            rc = L.gks_get_state(G._h, ptr(o[0]), ptr(o[1]), ptr(o[2]))
            assert rc == 0, gks.last_error()
        torch.cuda.synchronize()
        el_serial = time.perf_counter() - ts
        bytes_state = 3 * st.W.nbytes
        e2e = {"value": ncell * e_steps * ws / el, "unit": UNIT, "steps": e_steps,
               "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state,
               "api": "gks_step_host_async (pipelined), then gks_sync; median of 3 runs",
               "runs": [ncell * e_steps * ws / r for r in runs],
               "serial": {"value": ncell * e_steps * ws / el_serial,
                          "api": "gks_set_state + gks_step + gks_get_state per step"},
               "copy_gbs": pinned_copy_gbs(st.W.size * 3)}

    line = None
    if rank == 0:
        h = results[head]
        line = {"metric": metric_of(args), "value": h["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32-bulk (f64 time coefficients and accumulation)" if head == "fp32" else "f64",
                "data": "synthetic", "config": workload_config(args), "e2e": e2e,
                "gpu_launches": h["gpu_launches"], "roofline": h["roofline"], "clocks": h["clocks"],
                "kernel_ms_per_launch": h["kernel_ms_per_launch"],
                "alu_peaks_tflops": {"fp64": peaks["fp64"] / 1e12, "fp32": peaks["fp32"] / 1e12}}
        for form in forms:
            line[form] = results[form]
        if diff is not None:
            line["fp32_vs_fp64_l1_rho"] = diff
        if not args.no_cpu and ws == 1:
            keep = {}
            line["cpu_baseline"] = cpu_baseline(st, dt, keep=keep)
            try:
                line["cpu_baseline"]["single_thread"] = cpu_single_thread(st, dt)
            except Exception as e:  # an auxiliary figure: never lose the line over it
                line["cpu_baseline"]["single_thread"] = {"unavailable": f"{type(e).__name__}: {e}"}
            line["vs_oracle"] = vs_oracle(keep, dt, forms)
    G.close()

    # the other two workloads, as sub-objects of the same line
    if not args.no_sub and not shear:
        sh = inputs.shear_layer_2d(args.shear_n, order=8)
        sres, sdiff, (SG, _) = solver_workload(
            sh, ["fp32", "fp64"], {"fp32": args.shear_steps, "fp64": max(1, args.shear_steps // 3)},
            args.warmup, stream, local, dist, peaks, "wenoz_ns", 8, rank, True)
        SG.close()
        if line is not None:
            line["shear"] = {"metric": METRIC_SHEAR, "unit": UNIT,
                             "config": {"workload": f"shear_layer_2d_ns_{args.shear_n}x{args.shear_n}",
                                        "cells": args.shear_n ** 2, "order": 8, "recon": "wenoz",
                                        "mu": 1e-4, "Pr": 0.72, "cfl": CFL, "domain": "periodic [0,1]^2",
                                        "l2_policy": "inputs exceed L2"},
                             "value": sres["fp32"]["value"], "ms_per_step": sres["fp32"]["ms_per_step"],
                             "fp32": sres["fp32"], "fp64": sres["fp64"]}
        bres = batch_measure(args, ws, rank, local, dist, args.batch_steps)
        if line is not None:
            line["batch"] = bres
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
