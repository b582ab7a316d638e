"""Comparison rules between the CUDA path and the FP64 oracle.

FP64 rule (per output, per cell whose oracle status is 0):
  * |q_gpu - q_orc| <= 1e-10 |q_orc|   for rho, Z, cp, mu, lambda;
  * |h_gpu - h_orc| <= 1e-10 max(|h|, cp T)   (h crosses zero);
  * cells whose root condition number c = sum_k |c_k| |Z|^k / (|Z| |P'(Z)|)
    exceeds 1e4 (near-degenerate cubics: rounding of the coefficients moves
    the root by ~eps c) instead need |dZ|/Z <= 8 eps c, and rho, h, mu,
    lambda within 1e-10 + 100 * 8 eps c.  cp is not compared on these cells:
    it holds 1/(dp/dV)_T, which vanishes at the critical point, so its
    sensitivity to the root is unbounded there;
  * an output that misses 1e-10 on a well-conditioned root passes if the
    oracle shows it ill-conditioned in its inputs: with the componentwise
    condition number k_q = sum_x |d ln q / d ln x| over x in (T, p, Y_k)
    (central differences of the oracle), the bound is 1e-10 + 1e3 eps k_q.
    This covers Chung's correlations far outside their fitted range (e.g.
    H/H2-rich mixtures, whose G2 denominator E1 E4 + E2 + E3 is a difference
    of terms a thousand times larger);
  * cells the oracle flags ambiguous (two roots within 1e-9 in g_res) are
    excluded and counted; the GPU must flag them ok or ambiguous.
"""
import numpy as np

EPS = np.finfo(np.float64).eps
NAMES = ("rho", "Z", "h", "cp", "mu", "lambda")


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
    outputs with respect to relative perturbations of T, p and each Y_k."""
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


def assert_fp64_parity(gpu, gst, orc, ost, T, cond, rtol=1e-10, label="", kappa_fn=None):
    gpu = np.asarray(gpu, dtype=np.float64)
    ok = ost == 0
    amb = ost == 5
    assert np.all(np.isin(gst[amb], (0, 5))), f"{label}: ambiguous cells got status {np.unique(gst[amb])}"
    bad = (ost != 0) & (ost != 5)
    assert np.array_equal(gst[bad], ost[bad]), f"{label}: error statuses differ"
    assert np.all(np.isnan(gpu[:, bad])), f"{label}: error cells must be NaN"
    assert np.all(gst[ok] == 0), f"{label}: GPU status differs on {np.count_nonzero(gst[ok] != 0)} ok cells"
    err = rel_errors(gpu, orc, T)
    ill = cond > 1e4
    well = ok & ~ill
    worst = {}
    n_sens = 0
    if kappa_fn is not None:
        cand = np.nonzero(well & np.any(err > rtol, axis=0))[0]
        if cand.size:
            kap = kappa_fn(cand)
            tol = rtol + 1e3 * EPS * kap
            passed = np.all((err[:, cand] <= tol) | ~np.isfinite(tol), axis=0)
            well = well.copy()
            well[cand[passed]] = False
            n_sens = int(passed.sum())
    for q in range(6):
        e = err[q, well]
        worst[NAMES[q]] = float(e.max()) if e.size else 0.0
        if e.size and e.max() > rtol:
            i = np.nonzero(well)[0][int(np.argmax(e))]
            raise AssertionError(f"{label}: {NAMES[q]} rel err {e.max():.3e} > {rtol} at cell {i} "
                                 f"(T={T[i]}, gpu={gpu[q, i]!r}, orc={orc[q, i]!r}, cond={cond[i]:.3g})")
    sel = ok & ill
    if np.any(sel):
        tolZ = 8 * EPS * cond[sel]
        assert np.all(err[1, sel] <= np.maximum(tolZ, rtol)), f"{label}: ill-conditioned Z"
        for q in (0, 2, 4, 5):
            assert np.all(err[q, sel] <= rtol + 100 * tolZ), f"{label}: ill-conditioned {NAMES[q]}"
    return {"n_ok": int(well.sum()), "n_ill": int(sel.sum()), "n_ambiguous": int(amb.sum()),
            "n_input_ill_conditioned": n_sens, "max_rel": worst}


def error_summary(gpu, orc, T, mask):
    """Median, p99 and max relative error per output over `mask`."""
    err = rel_errors(np.asarray(gpu, dtype=np.float64), orc, T)
    out = {}
    for q in range(6):
        e = err[q, mask]
        out[NAMES[q]] = {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)), "max": float(e.max())}
    return out
