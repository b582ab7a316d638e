"""Train the surrogate on PR-labelled states and measure its error against the PR path.

Workload (the training configuration): a pool of states, half independent
uniform cells and half noisy flame-sheet states, labelled by the FP64
Peng-Robinson path (`pr_props`); states with non-physical outcomes dropped
(the paper's data constraints, Sec. 4.2); batches of 65536 drawn from the pool;
Adam with a cosine-decayed learning rate; error measured on held-out states
against the FP64 PR path.

    python -m paper_2312_04830_gb300.train --pool 67108864 --epochs 20 --save sg.ckpt

prints one JSON report.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import binding, workloads as W

OUT_NAMES = ("rho", "Z", "h", "cp", "mu", "lambda")
# physical-outcome filter: dense mu and lambda at least this fraction of their
# dilute-gas values at the same T and composition
DILUTE_FLOOR = 0.9


def label_pool(ctx, T, p, Y, device, chunk=1 << 23):
    """(x [11][n], y [6][n]) float32 device tensors of the physical states,
    labelled by the FP64 PR path, host arrays passed in pieces of `chunk`.

    Physical-outcome filter (the paper's data constraints, Sec. 4.2): positive
    finite properties, and a dense-fluid viscosity and conductivity of at least
    DILUTE_FLOOR times their dilute-gas values at the same T and composition
    (taken from the same path at p = 1 Pa).  Chung's dense correction,
    extrapolated to radical- and water-rich mixtures, can fall far below the
    dilute values or turn negative, where the excess viscosity of a gas is
    positive or, at high reduced temperature, only slightly negative; about
    1.7 % of the sampled states are dropped."""
    import torch
    xs, ys = [], []
    for a in range(0, T.size, chunk):
        b = min(T.size, a + chunk)
        d = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=device)
        Td, pd, Yd = d(T[a:b]), d(p[a:b]), d(Y[:, a:b])
        props, st = ctx.props(Td, pd, Yd, precision="fp64")
        dil, _ = ctx.props(Td, torch.ones_like(pd), Yd, precision="fp64", outputs=("mu", "lambda"))
        keep = (st == 0) & torch.all(torch.isfinite(props), dim=0) & torch.all(props[[0, 3, 4, 5]] > 0, dim=0)
        keep &= (props[4] >= DILUTE_FLOOR * dil[4]) & (props[5] >= DILUTE_FLOOR * dil[5])
        xs.append(torch.cat([Td[None], pd[None], Yd], dim=0)[:, keep].float())
        ys.append(props[:, keep].float())
    return torch.cat(xs, dim=1).contiguous(), torch.cat(ys, dim=1).contiguous()


INVERSE_OUT_NAMES = ("T", "rho", "psi", "mu", "alpha", "cp")


def label_pool_inverse(ctx, T, p, Y, device, chunk=1 << 23):
    """Pool of the inverse model (Sec. 4.1's arrangement): x = [h, p, Y] and
    y = [T, rho, psi, mu, alpha, cp], float32, from pr_props_ext in FP64 on the
    states (T, p, Y), with the same physical-outcome filter as label_pool and
    psi > 0 (a stable fluid's density rises with pressure at constant h)."""
    import torch
    xs, ys = [], []
    for a in range(0, T.size, chunk):
        b = min(T.size, a + chunk)
        d = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=device)
        Td, pd, Yd = d(T[a:b]), d(p[a:b]), d(Y[:, a:b])
        o, st = ctx.props_ext(Td, pd, Yd, precision="fp64")
        dil, _ = ctx.props(Td, torch.ones_like(pd), Yd, precision="fp64", outputs=("mu", "lambda"))
        keep = (st == 0) & torch.all(torch.isfinite(o), dim=0) & torch.all(o[[0, 3, 4, 5, 6, 7]] > 0, dim=0)
        keep &= (o[4] >= DILUTE_FLOOR * dil[4]) & (o[5] >= DILUTE_FLOOR * dil[5])
        xs.append(torch.cat([o[2][None], pd[None], Yd], dim=0)[:, keep].float())
        ys.append(torch.stack([Td, o[0], o[6], o[4], o[7], o[3]])[:, keep].float())
    return torch.cat(xs, dim=1).contiguous(), torch.cat(ys, dim=1).contiguous()


def label_pool_species(ctx, T, p, Y, device, kind, chunk=1 << 23):
    """Pool of a per-species network (the paper's diffusion and enthalpy
    networks, Sec. 4.1): x = [h, p, Y] from pr_props_ext in FP64, y = the 9
    D_k [m^2/s] (kind "dk") or h_k / (R T) ("hk") from pr_species_props at
    the states' T, float32; the same physical-outcome filter as label_pool."""
    import torch
    xs, ys = [], []
    for a in range(0, T.size, chunk):
        b = min(T.size, a + chunk)
        d = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=device)
        Td, pd, Yd = d(T[a:b]), d(p[a:b]), d(Y[:, a:b])
        o, st = ctx.props_ext(Td, pd, Yd, precision="fp64")
        dil, _ = ctx.props(Td, torch.ones_like(pd), Yd, precision="fp64", outputs=("mu", "lambda"))
        hk, dk, sst = ctx.species_props(Td, pd, Yd, precision="fp64")
        keep = (st == 0) & (sst == 0) & torch.all(torch.isfinite(o), dim=0) & torch.all(o[[0, 3, 4, 5, 6, 7]] > 0, dim=0)
        keep &= (o[4] >= DILUTE_FLOOR * dil[4]) & (o[5] >= DILUTE_FLOOR * dil[5])
        xs.append(torch.cat([o[2][None], pd[None], Yd], dim=0)[:, keep].float())
        ys.append((dk if kind == "dk" else hk)[:, keep].float())
    return torch.cat(xs, dim=1).contiguous(), torch.cat(ys, dim=1).contiguous()


def evaluate_field_species(sg, ctx, grid, device, kind):
    """Errors of a per-species network on the flame-vortex field against the
    FP64 per-species path at the field's T (relative RMS per species; h_k/(R T)
    relative to max(|h_k/(R T)|, 1))."""
    import torch
    T, p, Y = W.flame_vortex_field(grid)
    d64 = lambda v: torch.as_tensor(v, dtype=torch.float64, device=device)
    T64, p64, Y64 = d64(T), d64(p), d64(Y)
    o8, st = ctx.props_ext(T64, p64, Y64, precision="fp64")
    hk, dk, sst = ctx.species_props(T64, p64, Y64, precision="fp64")
    ref = dk if kind == "dk" else hk
    out, fb = sg.infer(o8[2].float(), p64.float(), Y64.float())
    ok = (st == 0) & (sst == 0)
    scale = ref.abs() if kind == "dk" else ref.abs().clamp_min(1.0)
    e = ((out.double() - ref) / scale)[:, ok]
    return {"cells": int(ok.sum()), "fallback_fraction": float(fb.float().mean()),
            "rel_rms": {nm: float(torch.sqrt(torch.mean(e[k] ** 2))) for k, nm in enumerate(W.SPECIES)},
            "p99": {nm: float(torch.quantile(e[k].abs()[:1 << 24].float(), 0.99)) for k, nm in enumerate(W.SPECIES)}}


def make_pool_inverse(ctx, n, seed, device):
    T, p, Y = W.training_states(n, seed=seed)
    return label_pool_inverse(ctx, T, p, Y, device)


def pool_states(n, seed, data="mixed", a2=20.0):
    """n states: "mixed" (half uniform cells, half noisy flame-sheet states),
    "manifold" (flame-sheet compositions with noisy T) or "augmented" (the
    paper's augmentation around the cells of a flame-vortex field)."""
    if data == "augmented":
        return W.augmented_field_states(n, seed=seed, a2=a2)
    if data == "manifold":
        return W.manifold_states(n, seed=seed, exact_frac=1.0)
    return W.training_states(n, seed=seed)


def make_pool(ctx, n, seed, device, data="mixed", a2=20.0):
    """Labelled forward-model pool of n states (see pool_states)."""
    T, p, Y = pool_states(n, seed, data, a2)
    return label_pool(ctx, T, p, Y, device)


def boxcox_lambda(z, shift, lo=-3.0, hi=3.0, iters=60):
    """Maximum-likelihood Box-Cox exponent of the values z + shift (golden
    section on the profile log-likelihood (lam - 1) sum log u - n/2 log var(BC))."""
    u = np.asarray(z, dtype=np.float64) + shift
    u = u[u > 0]
    lu = np.log(u)
    slu = lu.sum()

    def llf(lam):
        bc = lu if abs(lam) < 1e-12 else np.expm1(lam * lu) / lam
        return (lam - 1.0) * slu - 0.5 * u.size * np.log(bc.var())
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = llf(c), llf(d)
    for _ in range(iters):
        if fc > fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = llf(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = llf(d)
    return 0.5 * (a + b)


def evaluate_field_inverse(sg, ctx, grid, device):
    """Errors of an inverse-type surrogate (h, p, Y in; T, rho, psi, mu, alpha,
    cp out) on the flame-vortex field against the FP64 path at the field's T."""
    import torch
    T, p, Y = W.flame_vortex_field(grid)
    d64 = lambda v: torch.as_tensor(v, dtype=torch.float64, device=device)
    T64, p64, Y64 = d64(T), d64(p), d64(Y)
    o8, st = ctx.props_ext(T64, p64, Y64, precision="fp64")
    dil, _ = ctx.props(T64, torch.ones_like(p64), Y64, precision="fp64", outputs=("mu", "lambda"))
    out, fb = sg.infer(o8[2].float(), p64.float(), Y64.float())
    ref = torch.stack([T64, o8[0], o8[6], o8[4], o8[7], o8[3]])
    names = INVERSE_OUT_NAMES
    if out.shape[0] == 1:   # a dedicated single-property network
        j = binding.SINGLE_OUTPUTS.index(sg.single_output)
        ref, names = ref[j:j + 1], (INVERSE_OUT_NAMES[j],)
    ok = (st == 0) & torch.all(torch.isfinite(ref), dim=0)
    phys = ok & (o8[4] >= DILUTE_FLOOR * dil[4]) & (o8[5] >= DILUTE_FLOOR * dil[5])
    return {"cells": int(ok.sum()), "physical_cells": int(phys.sum()),
            "physical": relative_rms(out[:, phys], ref[:, phys].float(), names),
            "fallback_fraction": float(fb.float().mean())}


def evaluate_field(sg, ctx, grid, device):
    """Errors of the surrogate on the flame-vortex field against the FP64 PR
    path, on all cells and on the cells that pass the physical-outcome filter."""
    import torch
    T, p, Y = W.flame_vortex_field(grid)
    d64 = lambda v: torch.as_tensor(v, dtype=torch.float64, device=device)
    T64, p64, Y64 = d64(T), d64(p), d64(Y)
    ref, st = ctx.props(T64, p64, Y64, precision="fp64")
    dil, _ = ctx.props(T64, torch.ones_like(p64), Y64, precision="fp64", outputs=("mu", "lambda"))
    out, fb = sg.infer(T64.float(), p64.float(), Y64.float())
    ok = (st == 0) & torch.all(torch.isfinite(ref), dim=0)
    phys = ok & (ref[4] >= DILUTE_FLOOR * dil[4]) & (ref[5] >= DILUTE_FLOOR * dil[5])
    return {"cells": int(ok.sum()), "all": relative_rms(out[:, ok], ref[:, ok].float()),
            "physical_cells": int(phys.sum()), "physical": relative_rms(out[:, phys], ref[:, phys].float()),
            "fallback_fraction": float(fb.float().mean())}


def relative_rms(pred, ref, names=OUT_NAMES):
    """Per-output relative RMS error (h relative to max(|h|, std of h))."""
    import torch
    out = {}
    for j, nm in enumerate(names):
        s = torch.abs(ref[j])
        if nm == "h":
            s = torch.clamp(s, min=float(torch.std(ref[j])))
        e = (pred[j] - ref[j]) / s
        a = torch.abs(e[:1 << 24]).float()
        out[nm] = {"rel_rms": float(torch.sqrt(torch.mean(e * e))),
                   "p50": float(torch.quantile(a, 0.5)), "p99": float(torch.quantile(a, 0.99)),
                   "max": float(torch.max(torch.abs(e))), "frac_over_1pct": float(torch.mean((a > 0.01).float()))}
    return out


def evaluate(sg, x, y):
    """Errors of the surrogate (with its PR fallback) on held-out states."""
    import torch
    T, p, Y = x[0].contiguous(), x[1].contiguous(), x[2:]
    out, fb = sg.infer(T, p, Y)
    torch.cuda.synchronize()
    rep = {"all": relative_rms(out, y), "n": int(y.shape[1]), "fallback_fraction": float(fb.float().mean())}
    keep = fb == 0
    if int(keep.sum()) > 0:
        rep["surrogate_only"] = relative_rms(out[:, keep], y[:, keep])
    return rep


def train(sg, x, y, steps, batch=65536, lr0=1e-3, lr_min=1e-5, seed=20231207, log_every=1000):
    """Adam steps with a cosine-decayed learning rate; returns (losses, seconds)."""
    import torch
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(steps):
        lr = lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * s / max(1, steps)))
        sg.train_step(x, y, batch=batch, lr=lr, sample_seed=(seed << 20) + s + 1, loss_out=loss)
        if log_every and (s % log_every == 0 or s == steps - 1):
            losses.append((s, float(loss.item())))
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--pool", type=int, default=1 << 24)
    ap.add_argument("--heldout", type=int, default=1 << 20)
    ap.add_argument("--epochs", type=float, default=20.0)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--width", type=int, default=512)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--seed", type=int, default=20231207)
    ap.add_argument("--save", default=None)
    ap.add_argument("--loss", choices=("mse", "l1"), default="mse",
                    help="relative MSE on standardised targets, or the paper's L1 norm")
    ap.add_argument("--data", choices=("mixed", "manifold", "augmented"), default="mixed",
                    help="uniform + flame-sheet states, flame-sheet states, or the paper's augmentation around a field")
    ap.add_argument("--a2", type=float, default=20.0, help="divisor a2 of the augmentation")
    ap.add_argument("--eval-field", type=int, default=128, help="flame-vortex field edge for the field error")
    ap.add_argument("--model", choices=("forward", "inverse", "bilger"), default="forward",
                    help="T,p,Y -> properties; h,p,Y -> T and properties; or the same from h, p and Bilger's Z")
    ap.add_argument("--bc-shift", type=float, default=1e-3, help="Box-Cox shift of Bilger's Z")
    ap.add_argument("--outputs", choices=("props", "dk", "hk") + binding.SINGLE_OUTPUTS, default="props",
                    help="inverse / Bilger models: the six properties, the 9 D_k or h_k/(R T), "
                         "or one property alone (a dedicated network)")
    a = ap.parse_args()
    dev = torch.device("cuda:0")
    ctx = binding.PropertyContext(W.species_table())
    ctx.set_bilger(W.ATOMS_CHO, W.Y_FUEL, W.Y_OX)
    t0 = time.perf_counter()
    if a.model == "forward":
        x, y = make_pool(ctx, a.pool, a.seed, dev, a.data, a.a2)
        xh, yh = make_pool(ctx, a.heldout, a.seed + 1, dev)
    elif a.outputs in ("dk", "hk"):
        x, y = label_pool_species(ctx, *pool_states(a.pool, a.seed, a.data, a.a2), dev, a.outputs)
        xh, yh = None, None
    elif a.outputs != "props":   # one property of the inverse set
        x, y = label_pool_inverse(ctx, *pool_states(a.pool, a.seed, a.data, a.a2), dev)
        j = binding.SINGLE_OUTPUTS.index(a.outputs)
        y = y[j:j + 1].contiguous()
        xh, yh = None, None
    else:
        x, y = label_pool_inverse(ctx, *pool_states(a.pool, a.seed, a.data, a.a2), dev)
        xh, yh = label_pool_inverse(ctx, *pool_states(a.heldout, a.seed + 1, a.data, a.a2), dev)
    t_data = time.perf_counter() - t0
    sg = binding.Surrogate(ctx, width=a.width, hidden_layers=a.layers, max_batch=a.batch)
    bc = None
    if a.model != "forward":
        sg.set_mode(a.model)
    if a.outputs != "props":
        if a.model == "forward":
            raise SystemExit("per-species and single-property outputs need --model inverse or bilger")
        sg.set_outputs(a.outputs)
    if a.model == "bilger":
        z = ctx.bilger_z(x[2:, :1 << 20].contiguous(), precision="fp32").double().cpu().numpy()
        bc = boxcox_lambda(z, a.bc_shift)
        sg.set_boxcox(bc, a.bc_shift)
    sg.set_loss(a.loss)
    sg.fit_normalization(x, y)
    steps = int(round(a.epochs * x.shape[1] / a.batch))
    losses, secs = train(sg, x, y, steps, a.batch, a.lr, seed=a.seed)
    sg.sync_status()
    flops = 3 * 2 * (13 * a.width + (a.layers - 1) * a.width ** 2 + a.width * sg.n_out) * a.batch * steps
    rep = {"pool": int(x.shape[1]), "steps": steps, "batch": a.batch, "train_seconds": secs,
           "samples_per_s": steps * a.batch / secs, "train_tflops": flops / secs / 1e12,
           "data_seconds": t_data, "losses": losses, "loss": a.loss, "data": a.data, "model": a.model,
           "boxcox_lambda": bc}
    if a.model == "forward":
        rep["heldout"] = evaluate(sg, xh, yh)
    if a.eval_field > 0:
        if a.outputs in ("dk", "hk"):
            rep["field"] = evaluate_field_species(sg, ctx, a.eval_field, dev, a.outputs)
        elif a.model == "forward":
            rep["field"] = evaluate_field(sg, ctx, a.eval_field, dev)
        else:
            rep["field"] = evaluate_field_inverse(sg, ctx, a.eval_field, dev)
    rep["outputs"] = a.outputs
    if a.save:
        sg.save(a.save)
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
