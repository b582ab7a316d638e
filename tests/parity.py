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


def assert_fp64_parity(gpu, gst, orc, ost, T, cond, rtol=1e-10, label=""):
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
    return {"n_ok": int(well.sum()), "n_ill": int(sel.sum()), "n_ambiguous": int(amb.sum()), "max_rel": worst}


def error_summary(gpu, orc, T, mask):
    """Median, p99 and max relative error per output over `mask`."""
    err = rel_errors(np.asarray(gpu, dtype=np.float64), orc, T)
    out = {}
    for q in range(6):
        e = err[q, mask]
        out[NAMES[q]] = {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)), "max": float(e.max())}
    return out
