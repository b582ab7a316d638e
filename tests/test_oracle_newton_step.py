"""The error bound behind the FP64 inversion's one-step acceptance, checked on
the oracle (CPU).

On a smooth branch of h(T), one Newton step from T0 = T (1 + delta) lands at
T1 with |T1 - T| <= (kappa / 2) delta^2 T + |delta| eps_cp T, kappa =
T |dcp/dT| / cp, when the step divides by a cp with relative error eps_cp.  The
inversion takes such a step without a further evaluation when it is at most
1e-6 T, the state has one physical cubic root, cp is at most 3 times the
ideal-gas cp and no kink of h(T) (a NASA-7 range switch, the zero of a
species' alpha factor) lies near T, and it divides by the FP32 cp (eps_cp ~
2e-6).  Here the oracle's own h and cp make that step on uniform cells that
satisfy those conditions, and T1 must lie within the bound and far inside the
1e-10 parity tolerance.
"""
import numpy as np

from paper_2312_04830_gb300 import workloads as W


def _alpha_zero_T(species):
    """T at which 1 + kappa_k (1 - sqrt(T / Tc_k)) = 0, per species (Peng and
    Robinson's kappa(omega))."""
    w = np.asarray(species.omega, dtype=float)
    kap = 0.37464 + 1.54226 * w - 0.26992 * w * w
    return np.asarray(species.Tc, dtype=float) * ((1.0 + kap) / kap) ** 2


def test_one_newton_step_error_bound(orc, species):
    rng = np.random.default_rng(71)
    T, p, Y = W.uniform_cells(6000, seed=72)
    out, st, diag = orc.diagnose(species, T, p, Y)
    n_phys = np.array([d["n_phys"] for d in diag])
    dT = 1e-3 * T
    cp = out[3]
    cp_ig = (orc.h_ideal(species, T + dT, Y) - orc.h_ideal(species, T - dT, Y)) / (2 * dT)
    kinks = np.concatenate([np.asarray(species.T_mid, dtype=float), _alpha_zero_T(species)])
    clear = np.all(np.abs(T[:, None] - kinks[None, :]) > 1e-3 * T[:, None], axis=1)
    ok = (st == 0) & (n_phys == 1) & (cp <= 3.0 * cp_ig) & clear
    assert ok.sum() > 4000
    T, p, Y = T[ok], p[ok], Y[:, ok]
    hstar = out[2][ok]
    n = T.size
    delta = rng.choice([-1.0, 1.0], n) * rng.uniform(0.2, 1.0, n) * 1e-6
    eps_cp = rng.choice([-1.0, 1.0], n) * 2.3e-6
    T0 = T * (1.0 + delta)
    o0, s0 = orc.props(species, T0, p, Y)
    assert np.all(s0 == 0)
    T1 = T0 - (o0[2] - hstar) / (o0[3] * (1.0 + eps_cp))
    err = np.abs(T1 - T) / T
    # kappa from central differences of the oracle's cp
    hT = 1e-4 * T
    cpp, _ = orc.props(species, T + hT, p, Y)
    cpm, _ = orc.props(species, T - hT, p, Y)
    kappa = T * np.abs(cpp[3] - cpm[3]) / (2 * hT) / o0[3]
    bound = 0.5 * kappa * delta ** 2 + np.abs(delta) * np.abs(eps_cp) + 1e-14
    print("one-step error: max %.2e, kappa max %.1f, bound max %.2e" % (err.max(), kappa.max(), bound.max()))
    assert np.all(err <= 1.5 * bound)
    assert err.max() < 1e-10 / 10


def test_one_newton_step_error_grows_as_predicted(orc, species):
    """The same step from 1e-4 T away: the quadratic term dominates and the
    error scales with delta^2 -- the reason the acceptance stops at 1e-6 T."""
    T, p, Y = W.uniform_cells(2000, seed=73)
    out, st, diag = orc.diagnose(species, T, p, Y)
    n_phys = np.array([d["n_phys"] for d in diag])
    dT = 1e-3 * T
    cp_ig = (orc.h_ideal(species, T + dT, Y) - orc.h_ideal(species, T - dT, Y)) / (2 * dT)
    kinks = np.concatenate([np.asarray(species.T_mid, dtype=float), _alpha_zero_T(species)])
    clear = np.all(np.abs(T[:, None] - kinks[None, :]) > 2e-3 * T[:, None], axis=1)
    ok = (st == 0) & (n_phys == 1) & (out[3] <= 3.0 * cp_ig) & clear
    T, p, Y, hstar = T[ok], p[ok], Y[:, ok], out[2][ok]
    errs = []
    for delta in (1e-4, 1e-5):
        T0 = T * (1.0 + delta)
        o0, _ = orc.props(species, T0, p, Y)
        T1 = T0 - (o0[2] - hstar) / o0[3]
        errs.append(np.abs(T1 - T) / T)
    ratio = np.median(errs[0] / np.maximum(errs[1], 1e-300))
    print("error ratio for a 10x larger start: median %.1f" % ratio)
    assert 60.0 < ratio < 140.0       # ~100: quadratic convergence
    assert np.median(errs[0]) > 1e-10  # a start 1e-4 T away would not meet the parity bar in one step
