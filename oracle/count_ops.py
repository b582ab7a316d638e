"""Algorithmic FP64 work per cell of the forward property path, from the
oracle's operation counter (opcount.cpp) -- MEASUREMENT INFRASTRUCTURE.

    python -m oracle.count_ops [--grid 256] [--sample 65536]

Counts the oracle's per-cell operations on an evenly spaced sample of the
flame-vortex field, per step of the method (the oracle's own forms for the
composition, the root selection, the departures, Chung's dense correlation
and the output assembly; the exact short forms for the species terms, the
mixing sums, the cubic's roots, the ideal-gas sums and Chung's mixture
rules, see opcount.cpp), and weighs them into FP64 flops: an addition or
multiplication is one flop; a division, square root, cube root, exponential,
logarithm or power counts as the FP64-pipe work of one CUDA library call,
measured on GB300 by pr_measure_peak (DFMA slots per call, less the one extra
operation of the microbenchmark's chain, x 2 flops per slot).  Writes
oracle/op_counts_flame_vortex_<grid>.json.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

# FP64-pipe slots of one call (GB300, pr_measure_peak, bench pipe_peaks.fp64_call_slots,
# the chain's one extra operation subtracted): exp 19.0, log 37.0, div 6.75, sqrt 9.6,
# cbrt 17.3 measured; expm1 taken as exp, log1p as log, pow as log + exp, and the
# closed-form cubic's acos / cos as exp (none measured; the trigonometric seeds are
# 4 calls per three-root cell, 0.1 % of the field's cells)
CALL_SLOTS = {"div": 5.75, "sqrt": 8.6, "cbrt": 16.3, "exp": 18.0, "expm1": 18.0, "log": 36.0, "log1p": 36.0,
              "pow": 54.0, "trig": 18.0}
# steps taken as the oracle writes them, and the short forms that replace the others
LITERAL = ("composition", "root selection", "departures", "Chung dense correlation", "output assembly")
SHORT = ("species_terms", "mixing", "cubic_roots", "ideal_gas", "chung_rules")


def flops(kinds: dict) -> float:
    return kinds["add"] + kinds["mul"] + sum(2.0 * CALL_SLOTS[k] * kinds[k] for k in CALL_SLOTS)


def count(grid: int = 256, sample: int = 65536) -> dict:
    import oracle
    from paper_2312_04830_gb300 import workloads as W
    T, p, Y = W.flame_vortex_field(grid)
    idx = np.linspace(0, T.size - 1, sample).astype(np.int64)
    r = oracle.op_counts(W.species_table(), T[idx], p[idx], Y[:, idx])
    per_step = {s: r["steps"][s] for s in LITERAL}
    per_step.update({s: r["short"][s] for s in SHORT})
    steps_flops = {s: flops(k) for s, k in per_step.items()}
    calls = {k: sum(per_step[s][k] for s in per_step) for k in ("add", "mul", *CALL_SLOTS, "cmp")}
    return {"workload": f"flame-vortex field {grid}^3, {sample} cells evenly spaced", "cells": r["cells"],
            "call_slots": CALL_SLOTS, "per_step_counts": per_step, "per_step_flops": steps_flops,
            "operations_per_cell": calls, "fp64_flops_per_cell": sum(steps_flops.values()),
            "oracle_literal_counts": r["steps"], "short_form_check_max_rel": r["check"]}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--sample", type=int, default=65536)
    a = ap.parse_args()
    rep = count(a.grid, a.sample)
    path = os.path.join(HERE, f"op_counts_flame_vortex_{a.grid}.json")
    with open(path, "w") as f:
        json.dump(rep, f, indent=1)
    print(json.dumps({k: rep[k] for k in ("fp64_flops_per_cell", "per_step_flops", "operations_per_cell")}, indent=1))
