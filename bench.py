#!/usr/bin/env python
"""Throughput of the real-fluid property path on the 256^3 flame-vortex field.

One step = one pass of every path over the whole field, inputs resident in HBM:
  props_fp64   pr_props,    FP64           (rho, Z, h, cp, mu, lambda)
  newton_fp64  pr_T_from_h, FP64           (T from h* = h(T_true), start at T)
  props_fp32   pr_props,    FP32
  newton_fp32  pr_T_from_h, FP32
(+ surrogate paths when the library provides them).  `value` counts one
cell-evaluation per cell per path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  Under torchrun each rank evaluates its own
copy of the field (weak scaling, no collective on the data path).
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

METRIC = "cell-evals/s: PR FP64/FP32 vs BF16 MLP at <=1% rel err; %HBM roofline; p99 ms"
UNIT = "cell-evals/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (non-tensor), nominal

# Algorithmic bytes per cell of each path (N = 9 species): inputs + outputs
# that the path must move, FP64: T, p, Y[9] in, 6 outputs + int32 status out.
N_SPECIES = 9
BYTES_PER_CELL = {
    "props_fp64": (2 + N_SPECIES) * 8 + 6 * 8 + 4,
    "newton_fp64": (3 + N_SPECIES) * 8 + 8 + 4 + 4,
    "props_fp32": (2 + N_SPECIES) * 4 + 6 * 4 + 4,
    "newton_fp32": (3 + N_SPECIES) * 4 + 4 + 4 + 4,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--grid", type=int, default=256, help="field edge (cells = grid^3)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workload
def make_field(grid: int):
    from paper_2312_04830_gb300 import workloads as W
    T, p, Y = W.flame_vortex_field(grid)
    Ttrue = W.newton_targets(T)
    return T, p, Y, Ttrue


def cpu_baseline(T, p, Y, Ttrue, species, budget_cells_props=1 << 20, budget_cells_newton=1 << 18):
    """The FP64 oracle, as it stands, on the host cores over a bounded sample
    of the same field: props on the first cells, the inversion on the first
    cells of the perturbed-h workload (h* from the oracle itself)."""
    import oracle
    oracle.build()
    n1 = min(budget_cells_props, T.size)
    n2 = min(budget_cells_newton, T.size)
    # spread the sample over the field (every k-th cell) so that it spans all states
    s1 = np.linspace(0, T.size - 1, n1).astype(np.int64)
    s2 = np.linspace(0, T.size - 1, n2).astype(np.int64)
    tb = oracle.Table(species)
    t0 = time.perf_counter()
    oracle.props(tb, T[s1], p[s1], Y[:, s1])
    t1 = time.perf_counter()
    hs, _ = oracle.props(tb, Ttrue[s2], p[s2], Y[:, s2])
    t2 = time.perf_counter()
    oracle.T_from_h(tb, hs[2], p[s2], Y[:, s2], T[s2])
    t3 = time.perf_counter()
    secs = (t1 - t0) + (t3 - t2)
    return {"value": (n1 + n2) / secs, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"FP64 oracle: props on {n1} and T-from-h on {n2} cells spread evenly over the "
                      f"{T.size}-cell field; one cell-eval per cell per path",
            "seconds": secs}


# ----------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    from paper_2312_04830_gb300 import workloads as W
    import oracle
    oracle.build()
    T, p, Y, Ttrue = make_field(args.grid)
    species = W.species_table()
    tb = oracle.Table(species)
    n_props, n_newton = 1 << 17, 1 << 15
    s1 = np.linspace(0, T.size - 1, n_props).astype(np.int64)
    s2 = np.linspace(0, T.size - 1, n_newton).astype(np.int64)
    hs, _ = oracle.props(tb, Ttrue[s2], p[s2], Y[:, s2])

    def step():
        oracle.props(tb, T[s1], p[s1], Y[:, s1])
        oracle.T_from_h(tb, hs[2], p[s2], Y[:, s2], T[s2])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    secs = time.perf_counter() - t0
    v = (n_props + n_newton) * args.steps / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"flame-vortex field {args.grid}^3, FP64 oracle sample per step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"per step: props on {n_props} and T-from-h on {n_newton} cells spread "
                                       f"evenly over the field"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2312_04830_gb300 import binding, workloads as W

    species = W.species_table()
    ctx = binding.PropertyContext(species)
    T, p, Y, Ttrue = make_field(args.grid)
    n = T.size

    d64 = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    d32 = lambda a: torch.as_tensor(a, dtype=torch.float32, device=dev)
    T64, p64, Y64, Tt64 = d64(T), d64(p), d64(Y), d64(Ttrue)
    T32, p32, Y32, Tt32 = d32(T), d32(p), d32(Y), d32(Ttrue)
    # h* for the inversion: the FP64 path's own h at the perturbed T (set-up, untimed)
    hs64, _ = ctx.props(Tt64, p64, Y64, precision="fp64", outputs=("h",))
    hs64 = hs64[2].clone()
    hs32, _ = ctx.props(Tt32, p32, Y32, precision="fp32", outputs=("h",))
    hs32 = hs32[2].clone()
    out64 = torch.empty((6, n), dtype=torch.float64, device=dev)
    out32 = torch.empty((6, n), dtype=torch.float32, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    Tn64, Tn32 = torch.empty_like(T64), torch.empty_like(T32)
    it = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    paths = ["props_fp64", "newton_fp64", "props_fp32", "newton_fp32"]
    calls = {
        "props_fp64": lambda: ctx.props(T64, p64, Y64, "fp64", out=out64, status=st),
        "newton_fp64": lambda: ctx.T_from_h(hs64, p64, Y64, T64, "fp64", T_out=Tn64, status=st, iters=it),
        "props_fp32": lambda: ctx.props(T32, p32, Y32, "fp32", out=out32, status=st),
        "newton_fp32": lambda: ctx.T_from_h(hs32, p32, Y32, T32, "fp32", T_out=Tn32, status=st, iters=it),
    }
    launches_per_step = len(paths)

    def step(ev=None):
        for k, name in enumerate(paths):
            if ev is not None:
                ev[name][0].record(stream)
            calls[name]()
            if ev is not None:
                ev[name][1].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    evs = [{nm: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for nm in paths}
           for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index if ws == 1 else local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    t_start.record(stream)
    for s in range(args.steps):
        step(evs[s])
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    if ws > 1:
        tt = torch.tensor([elapsed_ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        elapsed_ms = float(tt.item())
    per_path_ms = {nm: statistics.mean(e[nm][0].elapsed_time(e[nm][1]) for e in evs) for nm in paths}
    evals = n * len(paths) * args.steps * ws
    value = evals / (elapsed_ms * 1e-3)

    # ----------------------------------------------------------- e2e
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(ctx, T, p, Y, Ttrue, hs64, hs32, dev, stream, max(2, min(args.steps, 4)), ws)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    pk, pk_kind = peaks()
    dom = max(per_path_ms, key=per_path_ms.get)
    roof_paths = {}
    for nm in paths:
        gbs = BYTES_PER_CELL[nm] * n / (per_path_ms[nm] * 1e-3) / 1e9
        roof_paths[nm] = {"ms": per_path_ms[nm], "cell_evals_per_s": n / (per_path_ms[nm] * 1e-3),
                          "algorithmic_GBps": gbs, "hbm_frac": gbs / pk["hbm_gbs"],
                          "bytes_per_cell": BYTES_PER_CELL[nm]}
    dom_gbs = roof_paths[dom]["algorithmic_GBps"]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": dom_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": dom_gbs / pk["hbm_gbs"], "traffic": None, "peak_source": pk_kind}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": f"flame-vortex field {args.grid}^3 = {n} cells, N=9 species, p = 10 MPa, "
                               "Burke-Schumann LOX/CH4 flame sheet on a Taylor-Green-distorted slab",
                   "cells": n, "paths": paths, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (FP64 inputs 1.5 GB per path call)"},
        "paths": roof_paths,
        "roofline": roofline,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(T, p, Y, Ttrue, species)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    ctx.close()
    return 0


def run_e2e(ctx, T, p, Y, Ttrue, hs64, hs32, dev, stream, steps, ws):
    """Same metric through the C ABI with HOST buffers: per step, pinned-host
    inputs are copied to the device, every path runs, and every output is
    copied back to pinned host memory."""
    import torch
    n = T.size
    pin = lambda a, dt: torch.as_tensor(a, dtype=dt).pin_memory()
    h_in64 = [pin(T, torch.float64), pin(p, torch.float64), pin(Y, torch.float64),
              hs64.cpu().pin_memory(), pin(T, torch.float64)]
    h_in32 = [pin(T, torch.float32), pin(p, torch.float32), pin(Y, torch.float32),
              hs32.cpu().pin_memory(), pin(T, torch.float32)]
    d_in64 = [torch.empty_like(x, device=dev) for x in h_in64]
    d_in32 = [torch.empty_like(x, device=dev) for x in h_in32]
    o64 = torch.empty((6, n), dtype=torch.float64, device=dev)
    o32 = torch.empty((6, n), dtype=torch.float32, device=dev)
    t64, t32 = torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.float32, device=dev)
    sts = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(4)]
    it = torch.empty(n, dtype=torch.int32, device=dev)
    h_out = [torch.empty((6, n), dtype=torch.float64).pin_memory(), torch.empty(n, dtype=torch.float64).pin_memory(),
             torch.empty((6, n), dtype=torch.float32).pin_memory(), torch.empty(n, dtype=torch.float32).pin_memory()]
    h_st = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(4)]
    d_out = [o64, t64, o32, t32]
    h2d = sum(x.numel() * x.element_size() for x in h_in64 + h_in32)
    d2h = sum(x.numel() * x.element_size() for x in h_out + h_st)

    def one():
        for h, d in zip(h_in64 + h_in32, d_in64 + d_in32):
            d.copy_(h, non_blocking=True)
        ctx.props(d_in64[0], d_in64[1], d_in64[2], "fp64", out=o64, status=sts[0])
        ctx.T_from_h(d_in64[3], d_in64[1], d_in64[2], d_in64[4], "fp64", T_out=t64, status=sts[1], iters=it)
        ctx.props(d_in32[0], d_in32[1], d_in32[2], "fp32", out=o32, status=sts[2])
        ctx.T_from_h(d_in32[3], d_in32[1], d_in32[2], d_in32[4], "fp32", T_out=t32, status=sts[3], iters=it)
        for d, h in zip(d_out + sts, h_out + h_st):
            h.copy_(d, non_blocking=True)

    one()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        one()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    if ws > 1:
        tt = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    return {"value": n * 4 * steps * ws / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
