"""Comparison rules between the CUDA path and the FP64 oracle.

FP64 rule (per output, per cell whose oracle status is 0):
  * |q_gpu - q_orc| <= 1e-10 |q_orc|   for rho, Z, cp, mu, lambda;
  * |h_gpu - h_orc| <= 1e-10 max(|h|, cp T)   (h crosses zero);
  * mu and lambda come out of sums that cancel for some mixtures far from
    Chung's fitted range (e.g. G2's denominator E1 E4 + E2 + E3 of H/H2-rich
    mixtures).  With c the cancellation ratio sum |t_i| / |sum t_i| of the
    worst such sum (the oracle reports it), terms that carry at most K_CHAIN
    roundings each (from the inputs through the mixture sums and the E_i, B_i
    coefficients) and the standard model of floating-point arithmetic, the
    computed sum is off by at most gamma(K_CHAIN) c of its value (Higham,
    Accuracy and Stability of Numerical Algorithms, Sec. 3.1 and 4.2); two
    such evaluations differ by at most twice that, so mu and lambda pass at
    1e-10 + 2 gamma(K_CHAIN) c;
  * cells whose root condition number c_Z = sum_k |c_k| |Z|^k / (|Z| |P'(Z)|)
    exceeds 1e4 (near-degenerate cubics: rounding of the coefficients moves
    the root by up to ~eps c_Z) need |dZ|/Z <= 8 eps c_Z, and every derived
    output is checked at the oracle's own root: it must lie within 1e-10 of
    its value plus twice the largest change that moving the oracle's root by
    that bound (8 eps c_Z, either way) causes in it;
  * cells the oracle flags ambiguous (two roots within 1e-9 in g_res) are
    excluded and counted; the GPU must flag them ok or ambiguous.
Every check reports how many cells each allowance took and asserts a
ceiling on them (0.1 % of the cells unless a test builds such cells on
purpose); the counts are summed in the run's terminal summary.
"""
import numpy as np

EPS = np.finfo(np.float64).eps
U = EPS / 2                 # unit roundoff of FP64
K_CHAIN = 35                # roundings per term of Chung's cancelling sums, the sum included
NAMES = ("rho", "Z", "h", "cp", "mu", "lambda")
COUNT_KEYS = ("n_cells", "n_ok", "n_ill", "n_ambiguous", "n_cancel")
REPORTS = []                # (label, counts) of every FP64 parity check of the run


def gamma(k):
    return k * U / (1 - k * U)


def cond_numbers(diags):
    return np.array([d["cond"] for d in diags])


def rel_errors(gpu, orc, T):
    """Relative error per output row, h scaled by max(|h|, cp T)."""
    err = np.empty_like(orc)
    for q in range(6):
        if NAMES[q] == "h":
            scale = np.maximum(np.abs(orc[2]), np.abs(orc[3]) * T)
        else:
            scale = np.abs(orc[q])
        err[q] = np.abs(gpu[q] - orc[q]) / scale
    return err


def input_condition(orc, species, T, p, Y, idx, h=1e-7):
    """Componentwise condition numbers k_q [6, len(idx)] of the oracle's
    outputs with respect to relative perturbations of T, p and each Y_k
    (a diagnostic of where an output is sensitive to its inputs)."""
    idx = np.asarray(idx)
    base, _ = orc.props(species, T[idx], p[idx], Y[:, idx])
    kap = np.zeros((6, idx.size))
    rows = [("T", None), ("p", None)] + [("Y", k) for k in range(Y.shape[0])]
    for which, k in rows:
        qs = []
        for sgn in (1.0, -1.0):
            Tt, pt, Yt = T[idx].copy(), p[idx].copy(), Y[:, idx].copy()
            if which == "T":
                Tt *= 1 + sgn * h
            elif which == "p":
                pt *= 1 + sgn * h
            else:
                Yt[k] *= 1 + sgn * h
            q, _ = orc.props(species, Tt, pt, Yt)
            qs.append(q)
        d = np.abs(qs[0] - qs[1]) / (2 * h * np.abs(base))
        kap += np.nan_to_num(d, nan=0.0, posinf=0.0)
    return kap


def root_sensitivity_bound(orc, species, T, p, Y, idx, Z, dz, o):
    """Largest change of each output [6, len(idx)] (relative, on the rule's
    scales) when the root of the cells idx moves from Z by dz (relative) either
    way: the outputs evaluated by the oracle at Z (1 +- dz)."""
    idx = np.asarray(idx)
    worst = np.zeros((6, idx.size))
    for sgn in (1.0, -1.0):
        q, _ = orc.props_at_Z(species, T[idx], p[idx], Y[:, idx], Z * (1 + sgn * dz))
        worst = np.maximum(worst, np.nan_to_num(rel_errors(q, o, T[idx]), nan=np.inf))
    return worst


def assert_fp64_parity(gpu, gst, orc_out, ost, T, diags, rtol=1e-10, label="", zsens=None,
                       max_frac=1e-3, expect_ill=False, expect_ambiguous=False):
    """FP64 parity by the rule above.  diags: the oracle's per-cell
    diagnostics (root condition number, Chung cancellation ratios, root);
    zsens(idx, Z, dz, o): root_sensitivity_bound for the cells idx (required
    when ill-conditioned roots occur).  Returns the counts."""
    gpu = np.asarray(gpu, dtype=np.float64)
    n = T.size
    cond = np.array([d["cond"] for d in diags])
    cmu = np.array([d["cancel_mu"] for d in diags])
    clam = np.array([d["cancel_lam"] for d in diags])
    Zo = np.array([d["Z"] for d in diags])
    ok = ost == 0
    amb = ost == 5
    assert np.all(np.isin(gst[amb], (0, 5))), f"{label}: ambiguous cells got status {np.unique(gst[amb])}"
    bad = (ost != 0) & (ost != 5)
    assert np.array_equal(gst[bad], ost[bad]), f"{label}: error statuses differ"
    assert np.all(np.isnan(gpu[:, bad])), f"{label}: error cells must be NaN"
    assert np.all(gst[ok] == 0), f"{label}: GPU status differs on {np.count_nonzero(gst[ok] != 0)} ok cells"
    err = rel_errors(gpu, orc_out, T)
    ill = cond > 1e4
    well = ok & ~ill
    tol = np.full(err.shape, rtol)
    tol[4] += 2 * gamma(K_CHAIN) * np.nan_to_num(cmu, nan=np.inf)
    tol[5] += 2 * gamma(K_CHAIN) * np.nan_to_num(clam, nan=np.inf)
    worst = {}
    for q in range(6):
        e = err[q, well]
        worst[NAMES[q]] = float(e.max()) if e.size else 0.0
        over = well & (err[q] > tol[q])
        if np.any(over):
            i = np.nonzero(over)[0][0]
            raise AssertionError(f"{label}: {NAMES[q]} rel err {err[q, i]:.3e} > {tol[q, i]:.3e} at cell {i} "
                                 f"(T={T[i]}, gpu={gpu[q, i]!r}, orc={orc_out[q, i]!r}, cond={cond[i]:.3g}, "
                                 f"cancel mu/lambda={cmu[i]:.3g}/{clam[i]:.3g})")
    n_cancel = int(np.count_nonzero(well & np.any(err > rtol, axis=0)))
    sel = ok & ill
    if np.any(sel):
        idx = np.nonzero(sel)[0]
        dz = 8 * EPS * cond[idx]
        assert np.all(err[1, idx] <= np.maximum(dz, rtol)), f"{label}: ill-conditioned Z"
        assert zsens is not None, f"{label}: ill-conditioned roots need the root-sensitivity bound"
        move = zsens(idx, Zo[idx], dz, orc_out[:, idx])
        for q in (0, 2, 3, 4, 5):
            lim = rtol + 2 * move[q]
            assert np.all(err[q, idx] <= lim), \
                f"{label}: ill-conditioned {NAMES[q]}: {err[q, idx].max():.3e} (limit {lim[np.argmax(err[q, idx])]:.3e})"
    counts = {"n_cells": int(n), "n_ok": int(np.count_nonzero(well)) - n_cancel, "n_ill": int(sel.sum()),
              "n_ambiguous": int(amb.sum()), "n_cancel": n_cancel}
    REPORTS.append((label, counts))
    print(f"FP64 parity {label}: {counts}")
    cap = max_frac * n
    assert n_cancel <= cap, f"{label}: {n_cancel} cells needed the cancellation allowance (ceiling {cap:g})"
    if not expect_ill:
        assert counts["n_ill"] <= cap, f"{label}: {counts['n_ill']} ill-conditioned roots (ceiling {cap:g})"
    if not expect_ambiguous:
        assert counts["n_ambiguous"] <= cap, f"{label}: {counts['n_ambiguous']} ambiguous cells (ceiling {cap:g})"
    return dict(counts, max_rel=worst)


def error_summary(gpu, orc, T, mask):
    """Median, p99 and max relative error per output over `mask`."""
    err = rel_errors(np.asarray(gpu, dtype=np.float64), orc, T)
    out = {}
    for q in range(6):
        e = err[q, mask]
        out[NAMES[q]] = {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)), "max": float(e.max())}
    return out
