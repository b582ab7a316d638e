#!/usr/bin/env python
"""Throughput of the real-fluid property path on the 256^3 flame-vortex field.

One step = one pass of every path over the whole field, inputs resident in HBM:
  props_fp64   pr_props,    FP64           (rho, Z, h, cp, mu, lambda)
  newton_fp64  pr_T_from_h, FP64           (T from h* = h(T_true), start at T)
  props_fp32   pr_props,    FP32
  newton_fp32  pr_T_from_h, FP32
  surrogate_bf16  surrogate_infer: BF16 tensor-core MLP, FP64 PR fallback
                  outside the training hull (trained first, untimed)
`value` counts one cell-evaluation per cell per path.

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
FALLBACK_BF16_TFLOPS_SUSTAINED = 1700.0
# FP64 (non-tensor) peak from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz;
# the roofline uses the DFMA throughput measured on the device (pr_measure_peak)
# when that succeeds, this nominal figure otherwise
FP64_PEAK_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = FP64_PEAK_NOMINAL_TFLOPS
# FP64 flops per cell the FP64 kernels execute, from ncu instruction counts
# (2 x DFMA + DADD + DMUL per launch / cells) of one launch on the 128^3
# flame-vortex field; reported beside the algorithmic count as kernel_flops
FP64_FLOPS_PER_CELL = {"props_fp64": 1413.5, "newton_fp64": 520.6, "species_fp64": 4117.0}
# Algorithmic FP64 work per cell of the forward property path, from the
# oracle's operation counter on the 256^3 flame-vortex field (oracle/count_ops.py,
# whose record is oracle/op_counts_flame_vortex_256.json): the method's
# additions and multiplications, with divisions, roots and transcendental calls
# weighted by the FP64-pipe work of one CUDA call measured on GB300.  The
# inversion's algorithmic work depends on how many evaluations a method takes,
# so its roofline stays on the executed count above.
ALGO_FP64_FLOPS_PER_CELL = {"props_fp64": 1698.6035400390624}
# DRAM bytes per cell (dram__bytes_read.sum + dram__bytes_write.sum per launch
# / cells) of the same captures; a full launch moves this x its cells (the
# forward surrogate: DRAM bytes per row of one resident-activation inference
# launch over a 2 Mi-row chunk of the 128^3 field)
TRAFFIC_BYTES_PER_CELL = {"props_fp64": 124.6, "newton_fp64": 125.4, "surrogate_bf16": 151.8}
# Instructions per cell the FP32 property kernel issues (ncu smsp__inst_executed.sum
# x 32 / cells, one full launch on the 128^3 flame-vortex field): the kernel is
# issue-bound, so its roofline is the issue rate, one warp instruction per
# clock per scheduler, 4 schedulers per SM
ISSUED_INSTR_PER_CELL = {"props_fp32": 1244.0}
# surrogate: 2 x (13*512 + 3*512^2 + 512*6) algorithmic flops per cell (4 x 512 hidden)
def mlp_flops_per_cell(width=512, layers=4, n_in=13, n_out=6):
    return 2.0 * (n_in * width + (layers - 1) * width * width + width * n_out)

# relative tolerance of the surrogates' transport test (mu, lambda against
# Chung's correlation at the network's own density; beyond it: FP64 fallback).
# The inverse model's fallback (an FP64 inversion) costs more per cell, and its
# network T enters the test, so it takes a wider tolerance.
TRANSPORT_CONFIDENCE = 0.02
TRANSPORT_CONFIDENCE_INVERSE = 0.05

# rows per surrogate inference chunk: all layers of a chunk run in one
# launch (CTA pairs with each 256-row block's activations in shared memory)
SG_CHUNK = 1 << 22

# Algorithmic bytes per cell of each path (N = 9 species): inputs + outputs
# that the path must move, FP64: T, p, Y[9] in, 6 outputs + int32 status out.
N_SPECIES = 9
BYTES_PER_CELL = {
    "props_fp64": (2 + N_SPECIES) * 8 + 6 * 8 + 4,
    "newton_fp64": (3 + N_SPECIES) * 8 + 8 + 4 + 4,
    "props_fp32": (2 + N_SPECIES) * 4 + 6 * 4 + 4,
    "newton_fp32": (3 + N_SPECIES) * 4 + 4 + 4 + 4,
    "surrogate_bf16": (2 + N_SPECIES) * 4 + 6 * 4 + 1,
    "surrogate_inverse_bf16": (2 + N_SPECIES) * 4 + 6 * 4 + 1,
    # per-species outputs: T, p, Y in; h_k/(R T) and D_k for every species + status out
    "species_fp64": (2 + N_SPECIES) * 8 + 2 * N_SPECIES * 8 + 4,
    "species_fp32": (2 + N_SPECIES) * 4 + 2 * N_SPECIES * 4 + 4,
    "props_mixed": (2 + N_SPECIES) * 4 + 6 * 4 + 4,
    "newton_mixed": (3 + N_SPECIES) * 4 + 4 + 4 + 4,
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
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--sg-pool", type=int, default=1 << 26, help="training states for the surrogate")
    ap.add_argument("--sg-epochs", type=float, default=20.0, help="epochs over the pool (batch 65536)")
    ap.add_argument("--sg-steps", type=int, default=0, help="Adam steps (overrides --sg-epochs when > 0)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-species", action="store_true", help="skip timing the per-species outputs")
    ap.add_argument("--serve-clients", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=16, help="requests per client")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_throughput(local_ms, units_per_rank, ws, device):
    """Whole-job throughput of a weak-scaling run: every rank processed
    units_per_rank units in local_ms; the job took the slowest rank's time.
    Returns (units of all ranks / s, max-over-ranks ms).  Collective over the
    default process group when ws > 1 (NCCL on the GPUs, gloo in the tests)."""
    ms = float(local_ms)
    if ws > 1:
        import torch
        tt = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    return units_per_rank * ws / (ms * 1e-3), ms


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


def cpu_baseline(T, p, Y, Ttrue, species, budget_cells_props=1 << 24, budget_cells_newton=1 << 22):
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
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.props(tb, T[s1], p[s1], Y[:, s1])
    t1 = time.perf_counter()
    hs, _ = oracle.props(tb, Ttrue[s2], p[s2], Y[:, s2])
    t2 = time.perf_counter()
    oracle.T_from_h(tb, hs[2], p[s2], Y[:, s2], T[s2])
    t3 = time.perf_counter()
    secs = (t1 - t0) + (t3 - t2)
    # one core on a 1/64 subsample of the same cells (per-core rate of the oracle)
    m1, m2 = s1[::64], s2[::64]
    t4 = time.perf_counter()
    oracle.props(tb, T[m1], p[m1], Y[:, m1], threads=1)
    t5 = time.perf_counter()
    oracle.T_from_h(tb, hs[2][::64], p[m2], Y[:, m2], T[m2], threads=1)
    t6 = time.perf_counter()
    return {"value": (n1 + n2) / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle: props on {n1} and T-from-h on {n2} cells spread evenly over the "
                      f"{T.size}-cell field; one cell-eval per cell per path",
            "seconds": secs,
            "single_core": {"value": (m1.size + m2.size) / (t6 - t4), "unit": UNIT, "cores": 1,
                            "sample": f"every 64th cell of the same samples ({m1.size} props, {m2.size} T-from-h)"}}


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
def train_surrogate(ctx, dev, args):
    """Train the surrogates on PR-labelled states (untimed set-up of the
    inference paths; their own throughput and held-out error are reported):
    the forward model and, on the same states, the inverse model."""
    import torch
    from paper_2312_04830_gb300 import binding, train as TR, workloads as W
    t0 = time.perf_counter()
    Tp, pp, Yp = W.training_states(args.sg_pool, seed=20231207)
    Th, ph, Yh = W.training_states(1 << 20, seed=20231208)
    x, y = TR.label_pool(ctx, Tp, pp, Yp, dev)
    xh, yh = TR.label_pool(ctx, Th, ph, Yh, dev)
    t_data = time.perf_counter() - t0
    pk, _ = peaks()
    bf16_peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops") or FALLBACK_BF16_TFLOPS_SUSTAINED
    sg = binding.Surrogate(ctx, width=512, hidden_layers=4, max_batch=65536, infer_chunk=SG_CHUNK)
    sg.fit_normalization(x, y)
    TR.train(sg, x, y, 20, 65536, 1e-3, log_every=0)          # warm-up steps
    sg.close()
    sg = binding.Surrogate(ctx, width=512, hidden_layers=4, max_batch=65536, infer_chunk=SG_CHUNK)
    sg.fit_normalization(x, y)
    # low-confidence cells take the FP64 fallback like cells outside the training hull:
    # predicted rho and Z off the equation of state by more than 1 %, or mu or lambda
    # more than 2 % away from Chung's correlation at the network's own density
    sg.set_confidence(0.01)
    sg.set_transport_confidence(TRANSPORT_CONFIDENCE)
    steps = args.sg_steps if args.sg_steps > 0 else int(round(args.sg_epochs * x.shape[1] / 65536))
    losses, secs = TR.train(sg, x, y, steps, 65536, 1e-3, log_every=max(1, steps // 10))
    sg.sync_status()
    flops = 3 * mlp_flops_per_cell() * 65536 * steps
    report = {"pool": int(x.shape[1]), "steps": steps, "batch": 65536, "seconds": secs,
              "samples_per_s": 65536 * steps / secs, "tflops": flops / secs / 1e12,
              "tensor_frac": flops / secs / 1e12 / bf16_peak,
              "epochs": 65536 * steps / x.shape[1], "data_seconds": t_data,
              "loss_first_last": [losses[0][1], losses[-1][1]],
              "heldout_error_vs_pr_fp64": TR.evaluate(sg, xh, yh)}
    del x, y, xh, yh
    # the inverse model (h, p, Y -> T, rho, psi, mu, alpha, cp), same recipe
    x, y = TR.label_pool_inverse(ctx, Tp, pp, Yp, dev)
    del Tp, pp, Yp
    sgi = binding.Surrogate(ctx, width=512, hidden_layers=4, max_batch=65536, infer_chunk=SG_CHUNK)
    sgi.set_mode("inverse")
    sgi.set_transport_confidence(TRANSPORT_CONFIDENCE_INVERSE)
    sgi.fit_normalization(x, y)
    steps_i = args.sg_steps if args.sg_steps > 0 else int(round(args.sg_epochs * x.shape[1] / 65536))
    losses_i, secs_i = TR.train(sgi, x, y, steps_i, 65536, 1e-3, log_every=max(1, steps_i // 10))
    sgi.sync_status()
    report["inverse"] = {"pool": int(x.shape[1]), "steps": steps_i, "seconds": secs_i,
                         "samples_per_s": 65536 * steps_i / secs_i,
                         "loss_first_last": [losses_i[0][1], losses_i[-1][1]]}
    del x, y
    return sg, sgi, report


def _latency_summary(lat, kinds, grids):
    """p50 / p99 [ms] overall, per request kind and per size class."""
    pct = lambda v: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99)), "n": int(v.size)} \
        if v.size else None
    out = {"all": pct(lat), "props": pct(lat[kinds == 0]), "T_from_h": pct(lat[kinds == 1])}
    for name, lo, hi in (("grid<=64", 0, 64), ("64<grid<=128", 64, 128), ("grid>128", 128, 1 << 30)):
        out[name] = pct(lat[(grids > lo) & (grids <= hi)])
    return out


def run_serving(ctx, sg, T, p, Y, hs64, args):
    """The serving workload: clients with flame-vortex fields of grid size
    log-uniform in [32, 256]^3 (sampled from the 256^3 field), 70 % forward
    properties / 30 % T-from-h, Poisson arrivals at twice the measured
    single-stream request rate, 80 GB admission budget.  The server's
    capacity is the request rate it sustains in that overloaded run; the
    same trace is then replayed at 0.5 and 0.8 of it, where queues stay
    bounded and p50/p99 measure the batching itself."""
    import torch
    from paper_2312_04830_gb300 import serving, workloads as W
    big = {"T": torch.as_tensor(T, dtype=torch.float32), "p": torch.as_tensor(p, dtype=torch.float32),
           "Y": torch.as_tensor(Y, dtype=torch.float32), "h": hs64.float().cpu()}
    g, kinds, clients = W.serving_trace(args.serve_clients, args.serve_requests)
    grid_of = {}
    for gi, c in zip(g, clients):
        grid_of.setdefault(int(c), int(gi))            # each client keeps its first grid size
    t0 = time.perf_counter()
    fields = {c: serving.client_field(big, gc) for c, gc in grid_of.items()}
    outs = {c: {"props": torch.empty((6, gc ** 3), dtype=torch.float32).pin_memory(),
                "T": torch.empty(gc ** 3, dtype=torch.float32).pin_memory(),
                "status": torch.empty(gc ** 3, dtype=torch.int32).pin_memory()} for c, gc in grid_of.items()}
    t_fields = time.perf_counter() - t0
    grids = np.array([grid_of[int(c)] for c in clients], dtype=np.int64)
    cells = grids ** 3
    srv = serving.Server(ctx, sg, chunk=1 << 18, max_slots=16, budget_bytes=80 << 30)
    # single-stream rate: requests of the trace served back to back, one at a time
    ns = min(32, len(g))
    t1 = time.perf_counter()
    for i in range(ns):
        c = int(clients[i])
        f, o = fields[c], outs[c]
        if kinds[i] == 0:
            tk = srv.submit_props(f["T"], f["p"], f["Y"], o["props"])
        else:
            tk = srv.submit_T_from_h(f["h"], f["p"], f["Y"], f["T"], o["T"], o["status"])
        st, res, _ = srv.wait(tk, 600000.0)
        assert st == 0 and res == 0
    single = (time.perf_counter() - t1) / ns
    rate = 2.0 / single
    arrivals = W.poisson_arrivals(len(g), rate)
    s0 = srv.stats()
    lat, makespan = serving.run_trace(srv, fields, g, kinds, clients.astype(np.int64), arrivals, outs)
    s1 = srv.stats()
    done_cells = int(cells.sum())
    capacity = len(g) / makespan                      # requests/s sustained when overloaded
    rep = {"clients": args.serve_clients, "requests": int(len(g)), "cells": done_cells,
           "frac_props": float(np.mean(kinds == 0)), "single_stream_s_per_request": single,
           "arrival_rate_per_s": rate, "makespan_s": makespan, "throughput_cells_per_s": done_cells / makespan,
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(lat.mean()), "max": float(lat.max())},
           "latency_ms_props_p99": float(np.percentile(lat[kinds == 0], 99)),
           "latency_ms_T_from_h_p99": float(np.percentile(lat[kinds == 1], 99)),
           "latency_ms_by_class": _latency_summary(lat, kinds, grids),
           "batches": int(s1["batches"] - s0["batches"]),
           "slot_fill": (s1["slots_used"] - s0["slots_used"]) / max(1, s1["slots_launched"] - s0["slots_launched"]),
           "peak_hbm_in_use_GB": s1["peak_bytes_in_use"] / 1e9, "budget_GB": 80 * 2 ** 30 / 1e9,
           "chunk": 1 << 18, "max_slots": 16, "host_field_setup_s": t_fields,
           "capacity_requests_per_s": capacity, "sustainable_load": {}}
    for frac in (0.5, 0.8):
        arr = W.poisson_arrivals(len(g), frac * capacity, seed=20231209)
        lat_f, mk = serving.run_trace(srv, fields, g, kinds, clients.astype(np.int64), arr, outs)
        rep["sustainable_load"][f"{frac}x_capacity"] = {
            "arrival_rate_per_s": frac * capacity, "makespan_s": mk, "throughput_cells_per_s": done_cells / mk,
            "latency_ms": _latency_summary(lat_f, kinds, grids)}
    srv.close()
    return rep


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
    # arithmetic-pipe peaks of this device (roofline denominators of the FP64 / FP32 paths)
    global FP64_PEAK_TFLOPS
    pipe_peaks = {"fp64_tflops_nominal": FP64_PEAK_NOMINAL_TFLOPS}
    try:
        pipe_peaks.update({"fp64_tflops": binding.measure_peak("fp64_fma") / 1e12,
                           "fp32_tflops": binding.measure_peak("fp32_fma") / 1e12,
                           "mufu_ex2_per_s": binding.measure_peak("mufu_ex2")})
        FP64_PEAK_TFLOPS = pipe_peaks["fp64_tflops"]
        pipe_peaks["fp64_source"] = "measured (pr_measure_peak, DFMA chains)"
        # FP64-pipe slots one call of CUDA's FP64 functions takes (DFMA rate / call rate)
        dfma_per_s = pipe_peaks["fp64_tflops"] * 1e12 / 2
        pipe_peaks["fp64_call_slots"] = {k: dfma_per_s / binding.measure_peak("fp64_" + k)
                                         for k in ("exp", "log", "div", "sqrt", "cbrt")}
    except binding.PrError as e:
        pipe_peaks["fp64_source"] = f"nominal (measurement failed: {e})"
    sg, sgi, sg_report = (None, None, None) if args.no_surrogate else train_surrogate(ctx, dev, args)
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
    del Tt64, Tt32
    out64 = torch.empty((6, n), dtype=torch.float64, device=dev)
    out32 = torch.empty((6, n), dtype=torch.float32, device=dev)
    outsg = torch.empty((6, n), dtype=torch.float32, device=dev)
    outsi = torch.empty((6, n), dtype=torch.float32, device=dev)
    fbi = torch.empty(n, dtype=torch.uint8, device=dev)
    # the inverse model's input: the field's own enthalpy (the flow's h, as the
    # paper's solver hands it over), from the FP64 path
    hT, _ = ctx.props(T64, p64, Y64, precision="fp64", outputs=("h",))
    hi32 = hT[2].float().contiguous()
    del hT
    fb = torch.empty(n, dtype=torch.uint8, device=dev)
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
    launches = {nm: 1 for nm in paths}
    if sg is not None:
        paths.append("surrogate_bf16")
        calls["surrogate_bf16"] = lambda: sg.infer(T32, p32, Y32, out=outsg, used_fallback=fb)
        n_chunks = (n + SG_CHUNK - 1) // SG_CHUNK
        launches["surrogate_bf16"] = n_chunks * (1 + 1 + 1 + 1)   # prep, MLP, confidence test, fallback
        # the inverse model: h*, p, Y -> T, rho, psi, mu, alpha, cp (the paper's arrangement)
        paths.append("surrogate_inverse_bf16")
        calls["surrogate_inverse_bf16"] = lambda: sgi.infer(hi32, p32, Y32, out=outsi, used_fallback=fbi)
        launches["surrogate_inverse_bf16"] = n_chunks * (1 + 1 + 1 + 1)   # prep, MLP, transport test, fallback
    launches_per_step = sum(launches.values())

    def step(ev=None):
        for name in paths:
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
    # the surrogates' MLP launches: CUDA events on the launching stream around
    # each chunk's MLP launch, inside surrogate_infer (SG_OPT_TIME_MLP)
    for m in (sg, sgi):
        if m is not None:
            m.set_time_mlp(True)
    barrier()
    t_start.record(stream)
    for s in range(args.steps):
        step(evs[s])
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    mlp_kernel = None
    if sg is not None:
        (mf, lf), (mi, li) = sg.mlp_time(), sgi.mlp_time()
        for m in (sg, sgi):
            m.set_time_mlp(False)
        rows = n * 2 * args.steps / (lf + li)
        mlp_kernel = {"kernel": {"resident": "mlp_resident_kernel", "single": "mlp_fused_kernel (single CTAs)",
                                 "pair": "mlp_fused_kernel (CTA pairs)", "per-layer": "gemm_kernel (per layer)"}[sg.fused_kind],
                      "launches_per_step": (lf + li) / args.steps, "rows_per_launch": rows,
                      "ms_per_launch": (mf + mi) / (lf + li), "ms_per_step": (mf + mi) / args.steps,
                      "forward_ms_per_step": mf / args.steps, "inverse_ms_per_step": mi / args.steps}
    value, elapsed_ms = job_throughput(t_start.elapsed_time(t_end), n * len(paths) * args.steps, ws, dev)
    per_path_ms = {nm: statistics.mean(e[nm][0].elapsed_time(e[nm][1]) for e in evs) for nm in paths}
    fb_frac = float(fb.float().mean()) if sg is not None else None

    # per-species outputs (h_k/(R T), mixture-averaged D_k) on the same field,
    # timed on their own after the step: they are not among the step's paths
    next_rows = None
    if not args.no_species:
        hk64, dk64 = (torch.empty((9, n), dtype=torch.float64, device=dev) for _ in range(2))
        hk32, dk32 = (torch.empty((9, n), dtype=torch.float32, device=dev) for _ in range(2))
        outm = torch.empty((6, n), dtype=torch.float32, device=dev)
        Tnm = torch.empty_like(T32)
        sp_calls = {
            "species_fp64": lambda: ctx.species_props(T64, p64, Y64, "fp64", hk=hk64, Dk=dk64, status=st),
            "species_fp32": lambda: ctx.species_props(T32, p32, Y32, "fp32", hk=hk32, Dk=dk32, status=st),
            # the mixed-precision pattern: FP32 arithmetic, FP64 where the root selection or
            # the pseudo-boiling inversion needs it
            "props_mixed": lambda: ctx.props(T32, p32, Y32, "mixed", out=outm, status=st),
            "newton_mixed": lambda: ctx.T_from_h(hs32, p32, Y32, T32, "mixed", T_out=Tnm, status=st, iters=it),
        }
        next_rows = {}
        for nm, fn in sp_calls.items():
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(args.steps, 3)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            r = {"ms": ms, "cell_evals_per_s": n / (ms * 1e-3), "bytes_per_cell": BYTES_PER_CELL[nm],
                 "algorithmic_GBps": BYTES_PER_CELL[nm] * n / (ms * 1e-3) / 1e9}
            if nm in FP64_FLOPS_PER_CELL:
                tf = FP64_FLOPS_PER_CELL[nm] * n / (ms * 1e-3) / 1e12
                r.update({"fp64_tflops": tf, "fp64_frac": tf / FP64_PEAK_TFLOPS})
            next_rows[nm] = r
        rel = lambda a, b: float(((a.double() - b).abs() / b.abs().clamp_min(1.0)).max())
        next_rows["species_fp32_max_rel_err_vs_fp64"] = {"hk_RT": rel(hk32, hk64),
                                                         "Dk": float(((dk32.double() - dk64).abs() / dk64).max())}
        from paper_2312_04830_gb300 import train as TR
        ok6 = torch.all(torch.isfinite(out64), dim=0) & torch.all(torch.isfinite(outm), dim=0)
        next_rows["props_mixed_error_vs_fp64"] = TR.relative_rms(outm[:, ok6], out64[:, ok6].float())
        del hk64, dk64, hk32, dk32, outm, Tnm

    # the FP64 inversion started from the inverse network's T (the surrogate as
    # the inversion's warm start), against the benchmark's start at the field's
    # T: FP64 Newton iterations per cell and time, with and without the FP32
    # warm start; results within the inversion's tolerance of each other
    warm = None
    if sgi is not None:
        outw = torch.empty((6, n), dtype=torch.float32, device=dev)
        fbw = torch.empty(n, dtype=torch.uint8, device=dev)
        sgi.infer(hs32, p32, Y32, out=outw, used_fallback=fbw)      # T from h* = h(T_true)
        Tnet = outw[0].double().contiguous()
        del outw
        ctx64 = binding.PropertyContext(species, newton_fp64_only=True)
        Tw = torch.empty_like(T64)
        warm = {"network_fallback_fraction": float(fbw.float().mean())}
        for name, c, guess in (("field_T_fp32_warm_start", ctx, T64), ("network_T_fp32_warm_start", ctx, Tnet),
                               ("field_T_fp64_only", ctx64, T64), ("network_T_fp64_only", ctx64, Tnet)):
            fn = lambda: c.T_from_h(hs64, p64, Y64, guess, "fp64", T_out=Tw, status=st, iters=it)
            for _ in range(2):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(3):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            okw = st == 0
            warm[name] = {"ms": e0.elapsed_time(e1) / 3, "fp64_iters_per_cell": float(it.double().mean()),
                          "converged_fraction": float(okw.double().mean()),
                          "max_rel_diff_vs_field_start": float(((Tw - Tn64).abs() / Tn64)[okw].max())}
        ctx64.close()
        del Tnet, Tw, fbw

    # error of the reduced-precision paths on the field against the FP64 PR
    # path's outputs of the last timed step (rel RMS, p99, max per property)
    field_err = None
    if rank == 0:
        from paper_2312_04830_gb300 import train as TR
        ref = out64.float()
        ok = torch.all(torch.isfinite(ref), dim=0)
        field_err = {"props_fp32": TR.relative_rms(out32[:, ok], ref[:, ok])}
        if sg is not None:
            field_err["surrogate_bf16"] = TR.relative_rms(outsg[:, ok], ref[:, ok])
            # the same on the cells that pass the training data's constraints
            # (dense mu, lambda at least TR.DILUTE_FLOOR of the dilute values)
            dil, _ = ctx.props(T64, torch.ones_like(p64), Y64, "fp64", outputs=("mu", "lambda"))
            phys = ok & (out64[4] >= TR.DILUTE_FLOOR * dil[4]) & (out64[5] >= TR.DILUTE_FLOOR * dil[5])
            del dil
            field_err["surrogate_bf16_physical"] = TR.relative_rms(outsg[:, phys], ref[:, phys])
            field_err["physical_cells"] = int(phys.sum())
            # inverse model against the field's T and pr_props_ext there (FP64), physical cells
            Tt64 = T64
            o8, st8 = ctx.props_ext(Tt64, p64, Y64, "fp64")
            dil, _ = ctx.props(Tt64, torch.ones_like(p64), Y64, "fp64", outputs=("mu", "lambda"))
            physi = (st8 == 0) & torch.all(torch.isfinite(o8), dim=0) & (o8[4] >= TR.DILUTE_FLOOR * dil[4]) & \
                (o8[5] >= TR.DILUTE_FLOOR * dil[5])
            refi = torch.stack([Tt64, o8[0], o8[6], o8[4], o8[7], o8[3]]).float()
            field_err["surrogate_inverse_bf16_physical"] = TR.relative_rms(outsi[:, physi], refi[:, physi],
                                                                           TR.INVERSE_OUT_NAMES)
            field_err["inverse_physical_cells"] = int(physi.sum())
            del o8, dil, refi, Tt64
        field_err["cells"] = int(ok.sum())

    # ----------------------------------------------------------- e2e
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(ctx, sg, sgi, hi32 if sgi is not None else None, T, p, Y, hs64, hs32, dev, stream,
                      max(2, min(args.steps, 4)), ws, ref64=out64)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    pk, pk_kind = peaks()
    bf16_peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops") or FALLBACK_BF16_TFLOPS_SUSTAINED
    roof_paths = {}
    for nm in paths:
        sec = per_path_ms[nm] * 1e-3
        gbs = BYTES_PER_CELL[nm] * n / sec / 1e9
        r = {"ms": per_path_ms[nm], "cell_evals_per_s": n / sec, "algorithmic_GBps": gbs,
             "hbm_frac": gbs / pk["hbm_gbs"], "bytes_per_cell": BYTES_PER_CELL[nm]}
        if nm in FP64_FLOPS_PER_CELL:
            fl = ALGO_FP64_FLOPS_PER_CELL.get(nm, FP64_FLOPS_PER_CELL[nm])
            tf = fl * n / sec / 1e12
            r.update({"fp64_tflops": tf, "fp64_frac": tf / FP64_PEAK_TFLOPS,
                      "fp64_flops_per_cell": fl,
                      "fp64_flops_source": "algorithmic (oracle op counter)" if nm in ALGO_FP64_FLOPS_PER_CELL
                      else "executed (ncu DFMA, DADD, DMUL counts)",
                      "kernel_flops_per_cell": FP64_FLOPS_PER_CELL[nm],
                      "kernel_fp64_frac": FP64_FLOPS_PER_CELL[nm] * n / sec / 1e12 / FP64_PEAK_TFLOPS})
        if nm in ISSUED_INSTR_PER_CELL:
            mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz")
            if mhz:
                issue_peak = 4 * torch.cuda.get_device_properties(dev).multi_processor_count * 32 * mhz * 1e6
                ir = ISSUED_INSTR_PER_CELL[nm] * n / sec
                r.update({"issued_instr_per_cell": ISSUED_INSTR_PER_CELL[nm], "thread_instr_per_s": ir,
                          "issue_frac": ir / issue_peak})
        if nm in ("surrogate_bf16", "surrogate_inverse_bf16"):
            ff = fb_frac if nm == "surrogate_bf16" else float(fbi.float().mean())
            tf = mlp_flops_per_cell() * n * (1.0 - ff) / sec / 1e12
            r.update({"tensor_tflops": tf, "tensor_frac": tf / bf16_peak, "fallback_fraction": ff})
        if nm == "surrogate_inverse_bf16":
            # the path it replaces: the FP64 inversion, then the FP64 properties
            r["speedup_vs_fp64_inversion_plus_props"] = (per_path_ms["newton_fp64"] +
                                                        per_path_ms["props_fp64"]) / per_path_ms[nm]
        roof_paths[nm] = r
    # the dominant kernel: the largest device time per step.  A PR path is one
    # kernel per call (its path time is the kernel's); the surrogates' MLP
    # launches are timed by their own events
    kernel_ms = {nm: per_path_ms[nm] for nm in paths if nm not in ("surrogate_bf16", "surrogate_inverse_bf16")}
    if mlp_kernel is not None:
        kernel_ms["mlp"] = mlp_kernel["ms_per_step"]
        tf = mlp_flops_per_cell() * mlp_kernel["rows_per_launch"] / mlp_kernel["ms_per_launch"] / 1e9
        mlp_kernel.update({"tensor_tflops": tf, "tensor_frac": tf / bf16_peak,
                           "traffic_per_launch": TRAFFIC_BYTES_PER_CELL["surrogate_bf16"] * mlp_kernel["rows_per_launch"]})
    dom = max(kernel_ms, key=kernel_ms.get)
    d = roof_paths.get(dom, {})
    if dom == "mlp":
        roofline = {"bound": "tensor", "kernel": mlp_kernel["kernel"], "achieved": mlp_kernel["tensor_tflops"],
                    "peak": bf16_peak, "unit": "TFLOP/s", "frac": mlp_kernel["tensor_frac"],
                    "traffic": mlp_kernel["traffic_per_launch"],
                    "flops_per_launch": mlp_flops_per_cell() * mlp_kernel["rows_per_launch"],
                    "ms_per_launch": mlp_kernel["ms_per_launch"],
                    "peak_source": f"{pk_kind} bf16 sustained",
                    "note": "algorithmic MLP flops of all rows of a launch (2 (13 x 512 + 3 x 512^2 + 512 x 6) "
                            "per row) / the launch's CUDA-event time; the PR FP64 property kernel's FP64-pipe "
                            "roofline is paths.props_fp64"}
    elif "fp64_tflops" in d:
        roofline = {"bound": "alu", "kernel": dom, "achieved": d["fp64_tflops"], "peak": FP64_PEAK_TFLOPS,
                    "peak_nominal": FP64_PEAK_NOMINAL_TFLOPS,
                    "unit": "TFLOP/s", "frac": d["fp64_frac"], "flops_per_cell": d["fp64_flops_per_cell"],
                    "flops_source": d["fp64_flops_source"], "kernel_frac": d["kernel_fp64_frac"],
                    "traffic": TRAFFIC_BYTES_PER_CELL[dom] * n if dom in TRAFFIC_BYTES_PER_CELL else None,
                    "peak_source": "FP64 pipe, " + pipe_peaks["fp64_source"] +
                                   "; nominal 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz"}
    elif "tensor_tflops" in d:
        roofline = {"bound": "tensor", "kernel": dom, "achieved": d["tensor_tflops"], "peak": bf16_peak,
                    "unit": "TFLOP/s", "frac": d["tensor_frac"],
                    "traffic": (TRAFFIC_BYTES_PER_CELL[dom] * min(SG_CHUNK, n)
                                if dom in TRAFFIC_BYTES_PER_CELL else None),
                    "peak_source": f"{pk_kind} bf16 sustained"}
    else:
        roofline = {"bound": "hbm", "kernel": dom, "achieved": d["algorithmic_GBps"], "peak": pk["hbm_gbs"],
                    "unit": "GB/s", "frac": d["hbm_frac"], "traffic": None, "peak_source": pk_kind}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32+bf16", "data": "synthetic",
        "config": {"workload": f"flame-vortex field {args.grid}^3 = {n} cells, N=9 species, p = 10 MPa, "
                               "Burke-Schumann LOX/CH4 flame sheet on a Taylor-Green-distorted slab",
                   "cells": n, "paths": paths, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (FP64 inputs 1.5 GB per path call)"},
        "paths": roof_paths,
        "field_error_vs_pr_fp64": field_err,
        "roofline": roofline,
        "mlp_kernel": mlp_kernel,
        "next_rows": next_rows,
        "inversion_from_network_T": warm,
        "pipe_peaks": pipe_peaks,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    if sg_report is not None:
        line["surrogate_training"] = sg_report
    if not args.no_serving and ws == 1:
        line["serving"] = run_serving(ctx, sg, T, p, Y, hs64, args)
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(T, p, Y, Ttrue, species)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    ctx.close()
    return 0


def run_e2e(ctx, sg, sgi, hi32, T, p, Y, hs64, hs32, dev, stream, steps, ws, n_chunks=8, n_slots=3, ref64=None):
    """Same metric through the C ABI with HOST buffers: per step, pinned-host
    inputs are copied to the device, every path runs, and every output is
    copied back to pinned host memory.  The field goes through in n_chunks
    pieces, pipelined over n_slots device buffer sets: the host-to-device
    copies of one piece (a copy stream), the six paths on another (the compute
    stream; the surrogates' internal buffers allow one call at a time) and the
    device-to-host copies of a third (a second copy stream) overlap."""
    import torch
    n = T.size
    cs = (n + n_chunks - 1) // n_chunks
    bounds = [(a, min(n, a + cs)) for a in range(0, n, cs)]
    pin = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
    hs64h, hs32h = hs64.cpu().numpy(), hs32.cpu().numpy()
    hi32h = hi32.cpu().numpy() if sgi is not None else None
    # host inputs, piece-major (each piece's Y block [9][len] contiguous, as a solver's
    # subdomain would hand it over)
    h_in = []
    for a, b in bounds:
        d = {"T64": pin(T[a:b], torch.float64), "p64": pin(p[a:b], torch.float64),
             "Y64": pin(Y[:, a:b], torch.float64), "hs64": pin(hs64h[a:b], torch.float64),
             "T32": pin(T[a:b], torch.float32), "p32": pin(p[a:b], torch.float32),
             "Y32": pin(Y[:, a:b], torch.float32), "hs32": pin(hs32h[a:b], torch.float32)}
        if sgi is not None:
            d["hi32"] = pin(hi32h[a:b], torch.float32)
        h_in.append(d)

    def out_set(m, device):
        o = {"o64": torch.empty((6, m), dtype=torch.float64, device=device),
             "t64": torch.empty(m, dtype=torch.float64, device=device),
             "o32": torch.empty((6, m), dtype=torch.float32, device=device),
             "t32": torch.empty(m, dtype=torch.float32, device=device)}
        for k in range(4):
            o[f"st{k}"] = torch.empty(m, dtype=torch.int32, device=device)
        if sg is not None:
            o["osg"] = torch.empty((6, m), dtype=torch.float32, device=device)
            o["fbd"] = torch.empty(m, dtype=torch.uint8, device=device)
        if sgi is not None:
            o["osi"] = torch.empty((6, m), dtype=torch.float32, device=device)
            o["fbi"] = torch.empty(m, dtype=torch.uint8, device=device)
        return o
    h_out = []
    for a, b in bounds:
        o = out_set(b - a, "cpu")
        h_out.append({k: v.pin_memory() for k, v in o.items()})
    slots = []
    for _ in range(n_slots):
        d_in = {k: torch.empty_like(v, device=dev) for k, v in h_in[0].items()}
        slots.append((d_in, out_set(cs, dev), torch.empty(cs, dtype=torch.int32, device=dev)))
    h2d = sum(v.numel() * v.element_size() for d in h_in for v in d.values())
    d2h = sum(v.numel() * v.element_size() for d in h_out for v in d.values())
    n_paths = 4 + (1 if sg is not None else 0) + (1 if sgi is not None else 0)
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event()
    e_in = [ev() for _ in range(n_slots)]
    e_comp = [ev() for _ in range(n_slots)]
    e_out = [ev() for _ in range(n_slots)]
    used = [False] * n_slots

    def piece(c, g):
        k = g % n_slots
        d_in, d_o, it = slots[k]
        m = bounds[c][1] - bounds[c][0]
        v = lambda t: t[..., :m]
        with torch.cuda.stream(s_in):
            if used[k]:
                s_in.wait_event(e_comp[k])                 # the slot's inputs are free again
            for key, h in h_in[c].items():
                (d_in[key][..., :m] if h.dim() == 2 else d_in[key][:m]).copy_(h, non_blocking=True)
            e_in[k].record(s_in)
        stream.wait_event(e_in[k])
        if used[k]:
            stream.wait_event(e_out[k])                    # the slot's outputs were read back
        T64, p64, Y64 = d_in["T64"][:m], d_in["p64"][:m], d_in["Y64"][:, :m]
        T32, p32, Y32 = d_in["T32"][:m], d_in["p32"][:m], d_in["Y32"][:, :m]
        ctx.props(T64, p64, Y64, "fp64", out=v(d_o["o64"]), status=d_o["st0"][:m], stream=stream)
        ctx.T_from_h(d_in["hs64"][:m], p64, Y64, T64, "fp64", T_out=d_o["t64"][:m], status=d_o["st1"][:m],
                     iters=it[:m], stream=stream)
        ctx.props(T32, p32, Y32, "fp32", out=v(d_o["o32"]), status=d_o["st2"][:m], stream=stream)
        ctx.T_from_h(d_in["hs32"][:m], p32, Y32, T32, "fp32", T_out=d_o["t32"][:m], status=d_o["st3"][:m],
                     iters=it[:m], stream=stream)
        if sg is not None:
            sg.infer(T32, p32, Y32, out=v(d_o["osg"]), used_fallback=d_o["fbd"][:m], stream=stream)
        if sgi is not None:
            sgi.infer(d_in["hi32"][:m], p32, Y32, out=v(d_o["osi"]), used_fallback=d_o["fbi"][:m], stream=stream)
        e_comp[k].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(e_comp[k])
            for key, h in h_out[c].items():
                h.copy_(v(d_o[key]), non_blocking=True)
            e_out[k].record(s_out)
        used[k] = True

    def one_step(g0):
        for c in range(len(bounds)):
            piece(c, g0 + c)
        return g0 + len(bounds)

    g = one_step(0)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s_in)
    for _ in range(steps):
        g = one_step(g)
    stream.wait_event(e_out[(g - 1) % n_slots])
    b.record(stream)
    torch.cuda.synchronize()
    value, ms = job_throughput(a.elapsed_time(b), n * n_paths * steps, ws, dev)
    rep = {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": steps,
           "pipeline": f"{len(bounds)} pieces per step over {n_slots} device buffer sets: "
                       "H2D copy stream, one compute stream, D2H copy stream"}
    if ref64 is not None:
        # the FP64 properties read back to the host equal the device-resident run's, bit for bit
        got = torch.cat([h["o64"] for h in h_out], dim=1)
        ref = ref64.cpu()
        rep["fp64_props_equal_device_run"] = bool(torch.all((got == ref) | (torch.isnan(got) & torch.isnan(ref))))
    return rep


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
