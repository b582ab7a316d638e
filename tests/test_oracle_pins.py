"""Pins of the FP64 oracle against what the paper and the mathematics fix.

CPU only.  Each test names the passage or the property it checks.  A plausible
mistake in the oracle (a dropped term, a wrong sign or index, a transposed
operand, a wrong constant) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2312_04830_gb300 import workloads as W

R = 8.314462618
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def one_hot(k, n=9):
    Y = np.zeros((n, 1))
    Y[k] = 1.0
    return Y


# ---------------------------------------------------------------- constants
def test_pr_constants_closed_form(orc):
    """Eq. 1: Omega_a, Omega_b at the critical point.  The oracle finds them
    by bisection on the critical-point condition; here they are checked
    against an independent closed form (Cardano on the eta-cubic) and against
    the five digits the paper prints."""
    Oa, Ob = orc.pr_constants()
    s8 = math.sqrt(8.0)
    eta = 1.0 / (1.0 + (4.0 - s8) ** (1.0 / 3.0) + (4.0 + s8) ** (1.0 / 3.0))
    assert Ob == pytest.approx(eta / (eta + 3.0), rel=1e-14)
    assert Oa == pytest.approx(8.0 * (5.0 * eta + 1.0) / (49.0 - 37.0 * eta), rel=1e-14)
    assert round(Oa, 5) == GOLDEN["pr_printed_Omega_a"]["value"]
    assert round(Ob, 5) == GOLDEN["pr_printed_Omega_b"]["value"]
    assert orc.pr_constants(printed=True) == (0.45724, 0.07780)


@pytest.mark.parametrize("k", range(6))
def test_pure_species_critical_Z(orc, species, k):
    """Eq. 1 at T = Tc, p = pc of a pure species: the triple root
    Z_c = 1/(3 + eta) = 0.3074013.  FP64 rounding spreads a triple root by
    ~eps^(1/3), so the tolerance is 1e-5."""
    out, st, d = orc.diagnose(species, [species.Tc[k]], [species.pc[k]], one_hot(k))
    zc = GOLDEN["pr_Zc_closed_form"]["value"]
    assert abs(d[0]["Z"] - zc) < 1e-5
    for r in d[0]["roots"][:d[0]["n_roots"]]:
        assert abs(r - zc) < 1e-5
    # A, B at the critical point equal Omega_a, Omega_b exactly (alpha(Tc) = 1)
    Oa, Ob = orc.pr_constants()
    assert d[0]["A"] == pytest.approx(Oa, rel=1e-13)
    assert d[0]["B"] == pytest.approx(Ob, rel=1e-13)


def test_printed_constants_have_no_triple_root(orc, species):
    """With the five-digit constants as printed, the cubic at the critical
    point keeps one real root near 0.3214 (the reason the exact values are
    used)."""
    t = orc.Table(species, printed_constants=True)
    out, st, d = orc.diagnose(t, [species.Tc[1]], [species.pc[1]], one_hot(1))
    assert d[0]["n_roots"] == 1
    assert d[0]["Z"] == pytest.approx(0.32138, abs=2e-5)


# ------------------------------------------------------------------- cubic
def _mp_real_roots(c2, c1, c0):
    import mpmath
    mpmath.mp.dps = 50
    rts = mpmath.polyroots([1, mpmath.mpf(c2), mpmath.mpf(c1), mpmath.mpf(c0)], maxsteps=200, extraprec=200)
    real = sorted(float(mpmath.re(r)) for r in rts if abs(mpmath.im(r)) <= mpmath.mpf(10) ** -30)
    cplx = [r for r in rts if abs(mpmath.im(r)) > mpmath.mpf(10) ** -30]
    min_im = min([abs(float(mpmath.im(r))) for r in cplx], default=math.inf)
    return real, min_im, rts


def test_cubic_roots_vs_high_precision(orc):
    """Every real root of the PR cubic (Eq. 1 in Z) against 50-digit
    polynomial roots of the same FP64 coefficients, over PR-shaped (A, B)."""
    rng = np.random.default_rng(7)
    checked3 = 0
    for _ in range(600):
        B = 10 ** rng.uniform(-3, -0.5)
        A = B * 10 ** rng.uniform(-0.5, 1.5)
        c2, c1, c0 = -(1 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)
        real, min_im, _ = _mp_real_roots(c2, c1, c0)
        if min_im < 1e-6:
            continue  # near a double root: classification is ill-posed in FP64
        rts = [r for r in real]
        if len(rts) > 1 and min(np.diff(rts)) < 1e-6:
            continue
        got = orc.cubic_real_roots(c2, c1, c0)
        assert len(got) == len(rts), (A, B, got, rts)
        for g, r in zip(got, rts):
            assert abs(g - r) <= 1e-13 * max(1.0, abs(r)) + 1e-15, (A, B, g, r)
        checked3 += len(rts) == 3
    assert checked3 > 50


def test_cubic_roots_vs_sign_scan(orc):
    """Brute force on tiny inputs: sign changes of P on a fine grid give the
    number of real roots and bracket each one."""
    rng = np.random.default_rng(11)
    grid = np.linspace(-2.0, 3.0, 500001)
    n3 = 0
    for _ in range(200):
        B = rng.uniform(0.01, 0.2)
        A = B * rng.uniform(1.0, 12.0)
        c2, c1, c0 = -(1 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)
        P = ((grid + c2) * grid + c1) * grid + c0
        sc = np.nonzero(np.sign(P[:-1]) * np.sign(P[1:]) < 0)[0]
        got = orc.cubic_real_roots(c2, c1, c0)
        if any(abs(P[i]) < 1e-9 or abs(P[i + 1]) < 1e-9 for i in sc):
            continue
        assert len(got) == len(sc), (A, B)
        for g, i in zip(got, sc):
            assert grid[i] <= g <= grid[i + 1]
        n3 += len(sc) == 3
    assert n3 > 10


def test_root_selection_minimum_gibbs(orc, species):
    """Root choice: among Z > B the root of least residual Gibbs energy.
    Brute force: evaluate g at every physical root and compare."""
    T, p, Y = W.uniform_cells(4096, seed=3)
    # plus subcritical pure H2O and CO2 states, where vapour- and liquid-like
    # physical roots coexist
    Tg, pg = np.meshgrid(np.linspace(0.55, 0.98, 20), np.linspace(0.05, 0.9, 20))
    for name in ("H2O", "CO2"):
        k = W.SPECIES.index(name)
        Yk = np.zeros((9, Tg.size))
        Yk[k] = 1.0
        T = np.concatenate([T, Tg.ravel() * species.Tc[k]])
        p = np.concatenate([p, pg.ravel() * species.pc[k]])
        Y = np.concatenate([Y, Yk], axis=1)
    out, st, d = orc.diagnose(species, T, p, Y)
    multi = 0
    for di in d:
        phys = [z for z in di["roots"][:di["n_roots"]] if z > di["B"]]
        if not phys:
            continue
        g = [orc.gres(z, di["A"], di["B"]) for z in phys]
        assert di["Z"] == phys[int(np.argmin(g))] or abs(max(g) - min(g)) < 1e-9
        multi += len(phys) > 1
    assert multi >= 100


# ------------------------------------------------------------ ideal limit
def test_low_pressure_limit(orc, species):
    """Z -> 1 and the departures vanish as p -> 0 (the ideal-gas model of
    the paper's ideal-gas cases, Sec. 2 and Table 1)."""
    T, _, Y = W.uniform_cells(2000, seed=5)
    # above every critical temperature: at 1 Pa and low T the condensed root of
    # H2O-rich mixtures is the stable one (its vapour pressure is below 1 Pa)
    T = 700.0 + (T - 100.0) * (2800.0 / 3400.0)
    p = np.full(T.size, 1.0)
    out, st, d = orc.diagnose(species, T, p, Y)
    assert np.all(st == 0)
    for i, di in enumerate(d):
        assert abs(di["Z"] - 1.0) < 1e-6
        assert abs(di["h_dep"]) / (R * T[i]) < 1e-6
        assert abs(di["cp_dep"]) / R < 1e-6
        assert out[0, i] == pytest.approx(p[i] * di["Wbar"] / (R * T[i]), rel=1e-6)
        assert out[2, i] == pytest.approx(di["h_ig"], abs=1e-6 * max(abs(di["h_ig"]), di["cp_ig"] * T[i]))
        # Chung: the dense correction vanishes with the density.  The dense
        # form's prefactor 36.344 sqrt(1.2593) and the dilute 40.785 are both
        # published to 5 digits and agree to 5e-6.
        assert out[4, i] == pytest.approx(di["mu_dilute"], rel=1e-5)
        assert out[5, i] == pytest.approx(di["lambda_dilute"], rel=1e-6)


def test_h_ideal_is_the_low_pressure_enthalpy(orc, species):
    """The batch ideal-gas enthalpy (the surrogate's exact part) equals the
    full enthalpy in the p -> 0 limit and the per-cell diagnostic h_ig, on
    uniform and flame-sheet states, both NASA ranges."""
    T, _, Y = W.uniform_cells(400, seed=6)
    T = 700.0 + (T - 100.0) * (2800.0 / 3400.0)
    Tm, _, Ym = W.manifold_states(400, seed=7)
    T, Y = np.concatenate([T, np.maximum(Tm, 700.0)]), np.concatenate([Y, Ym], axis=1)
    hig = orc.h_ideal(species, T, Y)
    out, st, d = orc.diagnose(species, T, np.full(T.size, 1e-3), Y)
    assert np.all(st == 0)
    scale = np.maximum(np.abs(out[2]), out[3] * T)
    assert np.all(np.abs(hig - out[2]) <= 1e-9 * scale)
    assert np.array_equal(hig, np.array([di["h_ig"] for di in d]))


# JANAF / CODATA standard enthalpies of formation at 298.15 K [kJ/mol] and
# ideal-gas cp [J/(mol K)]; checks the NASA-7 evaluation (and the data).
HF298 = {"CH4": -74.6, "O2": 0.0, "CO2": -393.51, "H2O": -241.83, "CO": -110.53, "H2": 0.0,
         "H": 218.0, "O": 249.18}
CP298 = {"CH4": 35.69, "O2": 29.38, "CO2": 37.12, "H2O": 33.59, "CO": 29.14, "H2": 28.84,
         "H": 20.786, "O": 21.91}


@pytest.mark.parametrize("name", list(HF298))
def test_ideal_gas_reference_state(orc, species, name):
    k = W.SPECIES.index(name)
    out, st, d = orc.diagnose(species, [298.15], [1.0], one_hot(k))
    Wk = species.W[k] * 1e-3
    assert d[0]["h_ig"] * Wk / 1e3 == pytest.approx(HF298[name], abs=0.3)
    assert d[0]["cp_ig"] * Wk == pytest.approx(CP298[name], rel=3e-3)


def test_nasa7_data_continuity(species):
    """Data quality: cp, h and s of each two-range set agree at T_mid."""
    for k in range(species.n):
        lo, hi, T = species.nasa_lo[k], species.nasa_hi[k], species.T_mid[k]
        cp = lambda a: a[0] + a[1] * T + a[2] * T ** 2 + a[3] * T ** 3 + a[4] * T ** 4
        h = lambda a: a[0] + a[1] * T / 2 + a[2] * T ** 2 / 3 + a[3] * T ** 3 / 4 + a[4] * T ** 4 / 5 + a[5] / T
        s = lambda a: a[0] * np.log(T) + a[1] * T + a[2] * T ** 2 / 2 + a[3] * T ** 3 / 3 + a[4] * T ** 4 / 4 + a[6]
        assert abs(cp(lo) - cp(hi)) < 1e-6
        assert abs(h(lo) - h(hi)) < 1e-6
        assert abs(s(lo) - s(hi)) < 1e-6
    kH = W.SPECIES.index("H")
    assert species.nasa_lo[kH][0] == 2.5


# ------------------------------------------------------- cp = dh/dT, a_m
def _kink_temperatures(species):
    """alpha's inner factor 1 + kappa (1 - sqrt(T/Tc)) vanishes at
    T* = Tc (1 + 1/kappa)^2; a_m has a kink there."""
    w = species.omega
    kap = 0.37464 + 1.54226 * w - 0.26992 * w * w
    return species.Tc * (1.0 + 1.0 / kap) ** 2


def _fd_ok(T, delta, species, d_list):
    tstars = _kink_temperatures(species)
    if np.any(np.abs(T - tstars) < 4 * delta):
        return False
    if abs(T - 1000.0) < 4 * delta:
        return False
    return all(di["n_phys"] == 1 and di["cond"] < 1e3 for di in d_list)


def test_cp_equals_dh_dT(orc, species):
    """cp from the PR departure formulas equals the Richardson-extrapolated
    central difference of h(T) at fixed p, Y (consistency of h and cp)."""
    T, p, Y = W.uniform_cells(600, seed=9)
    n_checked = 0
    for i in range(T.size):
        Ti, d0 = T[i], 1e-4 * T[i]
        Ts = np.array([Ti, Ti - d0, Ti + d0, Ti - d0 / 2, Ti + d0 / 2])
        Yi = np.repeat(Y[:, i:i + 1], 5, axis=1)
        out, st, d = orc.diagnose(species, Ts, np.full(5, p[i]), Yi)
        if not np.all(st == 0) or not _fd_ok(Ti, d0, species, d):
            continue
        h = out[2]
        D1 = (h[2] - h[1]) / (2 * d0)
        D2 = (h[4] - h[3]) / d0
        Rich = (4 * D2 - D1) / 3
        assert Rich == pytest.approx(out[3, 0], rel=1e-6), (Ti, p[i])
        # a_m derivatives
        am = np.array([di["am"] for di in d])
        dam = (4 * (am[4] - am[3]) / d0 - (am[2] - am[1]) / (2 * d0)) / 3
        d2am = (am[2] - 2 * am[0] + am[1]) / d0 ** 2
        assert dam == pytest.approx(d[0]["dam"], rel=1e-7, abs=1e-9 * abs(d[0]["am"]) / Ti)
        assert d2am == pytest.approx(d[0]["d2am"], rel=1e-4, abs=1e-6 * abs(d[0]["am"]) / Ti ** 2)
        n_checked += 1
    assert n_checked > 400


def test_flame_field_cp_fd(orc, species):
    """The same consistency on flame-sheet states (pure LOX at 120 K, CH4 at
    300 K and hot products)."""
    Zm = np.linspace(0.0, 1.0, 101)
    T, Y = W.flame_sheet_state(Zm)
    n = 0
    for i in range(T.size):
        Ti, d0 = T[i], 1e-4 * T[i]
        Ts = np.array([Ti, Ti - d0, Ti + d0, Ti - d0 / 2, Ti + d0 / 2])
        out, st, d = orc.diagnose(species, Ts, np.full(5, 10e6), np.repeat(Y[:, i:i + 1], 5, axis=1))
        if not np.all(st == 0) or not _fd_ok(Ti, d0, species, d):
            continue
        h = out[2]
        Rich = (4 * (h[4] - h[3]) / d0 - (h[2] - h[1]) / (2 * d0)) / 3
        assert Rich == pytest.approx(out[3, 0], rel=1e-6)
        n += 1
    assert n > 80


def test_mechanical_stability(orc, species):
    T, p, Y = W.uniform_cells(4096, seed=13)
    out, st, d = orc.diagnose(species, T, p, Y)
    for i, di in enumerate(d):
        if st[i] != 0:
            continue
        assert di["Z"] > di["B"]
        assert out[0, i] > 0
        if di["n_phys"] == 1:
            assert di["dpdV"] < 0


# ------------------------------------------------------------- mixing
def test_mixing_permutation_invariance(orc, species):
    T, p, Y = W.uniform_cells(512, seed=17)
    perm = np.array([4, 7, 0, 2, 8, 1, 6, 3, 5])
    names = [W.SPECIES[k] for k in perm]
    sp2 = W.SpeciesTable(names)
    o1, s1 = orc.props(species, T, p, Y)
    o2, s2 = orc.props(sp2, T, p, Y[perm])
    ok = (s1 == 0) & (s2 == 0)
    assert ok.sum() > 500
    np.testing.assert_allclose(o2[:, ok], o1[:, ok], rtol=1e-11, atol=0)


@pytest.mark.parametrize("name", ["CH4", "O2", "CO2", "H2O", "H2"])
def test_one_hot_equals_pure(orc, species, name):
    """A one-hot mixture equals the single-component evaluation, for both
    transport rules (Chung's mixing rules reduce to the pure fluid)."""
    k = W.SPECIES.index(name)
    pure = W.SpeciesTable([name])
    T = np.linspace(120.0, 3000.0, 57)
    Ymix = np.zeros((9, T.size))
    Ymix[k] = 1.0
    o1, s1 = orc.props(species, T, 10e6, Ymix)
    o2, s2 = orc.props(pure, T, 10e6, np.ones((1, T.size)))
    o3, s3 = orc.props(species, T, 10e6, Ymix, transport_rule=1)
    np.testing.assert_allclose(o1, o2, rtol=1e-12)
    np.testing.assert_allclose(o3, o2, rtol=1e-12)


def test_duplicate_species_split(orc, species):
    """Splitting a species into two identical entries changes nothing."""
    T, p, Y = W.uniform_cells(256, seed=19)
    names = list(W.SPECIES) + ["O2"]
    sp2 = W.SpeciesTable(names)
    Y2 = np.vstack([Y, np.zeros((1, T.size))])
    Y2[1] = 0.3 * Y[1]
    Y2[9] = 0.7 * Y[1]
    o1, s1 = orc.props(species, T, p, Y)
    o2, s2 = orc.props(sp2, T, p, Y2)
    ok = (s1 == 0) & (s2 == 0)
    np.testing.assert_allclose(o2[:, ok], o1[:, ok], rtol=1e-12)


def test_kij_enters_as_pair_weight(orc, species):
    """Brute force on a 2-species mixture: a_m = X1^2 a1 + X2^2 a2 +
    2 X1 X2 (1 - k12) sqrt(a1 a2)."""
    sp0 = W.SpeciesTable(["CH4", "O2"])
    k12 = 0.1
    sp1 = W.SpeciesTable(["CH4", "O2"], kij=np.array([[0.0, k12], [k12, 0.0]]))
    Y = np.array([[0.3], [0.7]])
    T = [250.0]
    _, _, d0 = orc.diagnose(sp0, T, [10e6], Y)
    _, _, d1 = orc.diagnose(sp1, T, [10e6], Y)
    _, _, dA = orc.diagnose(W.SpeciesTable(["CH4"]), T, [10e6], np.ones((1, 1)))
    _, _, dB = orc.diagnose(W.SpeciesTable(["O2"]), T, [10e6], np.ones((1, 1)))
    x1 = (0.3 / 16.043) / (0.3 / 16.043 + 0.7 / 31.998)
    x2 = 1 - x1
    a1, a2 = dA[0]["am"], dB[0]["am"]
    cross = 2 * x1 * x2 * math.sqrt(a1 * a2)
    assert d0[0]["am"] == pytest.approx(x1 * x1 * a1 + x2 * x2 * a2 + cross, rel=1e-13)
    assert d1[0]["am"] == pytest.approx(x1 * x1 * a1 + x2 * x2 * a2 + (1 - k12) * cross, rel=1e-13)
    assert d0[0]["bm"] == pytest.approx(x1 * dA[0]["bm"] + x2 * dB[0]["bm"], rel=1e-14)


def test_alpha_kink_uses_abs(orc, species):
    """Above T* = Tc (1 + 1/kappa)^2 the inner factor of alpha changes sign;
    sqrt(a_i a_j) stays non-negative so a_m of a one-hot mixture keeps
    growing as a_c u^2 (no sign flip of the cross term)."""
    k = W.SPECIES.index("CO")
    ts = _kink_temperatures(species)[k]
    Ts = np.array([0.9 * ts, ts * 1.1])
    _, _, d = orc.diagnose(species, Ts, np.full(2, 10e6), np.repeat(one_hot(k), 2, axis=1))
    Oa, _ = orc.pr_constants()
    kap = 0.37464 + 1.54226 * species.omega[k] - 0.26992 * species.omega[k] ** 2
    for T, di in zip(Ts, d):
        u = 1 + kap * (1 - math.sqrt(T / species.Tc[k]))
        ac = Oa * R * R * species.Tc[k] ** 2 / species.pc[k]
        assert di["am"] == pytest.approx(ac * u * u, rel=1e-13)


# ---------------------------------------------------------------- Newton
def test_newton_inverts_h(orc, species):
    """T(h(T), p, Y) = T on the uniform workload (the solver's T-from-h step,
    Sec. 4.1)."""
    T, p, Y = W.uniform_cells(2048, seed=23)
    out, st = orc.props(species, T, p, Y)
    guess = T * (1 + np.random.default_rng(1).uniform(-0.05, 0.05, T.size))
    Tout, st2, it = orc.T_from_h(species, out[2], p, Y, guess)
    ok = (st == 0) & (st2 == 0)
    assert ok.sum() > 2000
    np.testing.assert_allclose(Tout[ok], T[ok], rtol=1e-11)
    assert np.all(it[ok] <= 60)


def test_newton_status_codes(orc, species):
    T = np.array([300.0, 300.0, 300.0])
    Y = np.zeros((9, 3))
    Y[0] = 1.0
    hlow = -1e9
    hhigh = 1e9
    Tout, st, it = orc.T_from_h(species, np.array([hlow, hhigh, np.nan]), np.full(3, 10e6), Y, T)
    assert list(st) == [2, 2, 4]
    assert Tout[0] == 60.0 and Tout[1] == 5000.0


def test_bad_inputs_flagged(orc, species):
    T = np.array([300.0, -1.0, np.nan, 300.0, 300.0])
    p = np.array([1e7, 1e7, 1e7, -5.0, 1e7])
    Y = np.zeros((9, 5))
    Y[1] = 1.0
    Y[1, 4] = 0.9   # sum off by 0.1
    out, st = orc.props(species, T, p, Y)
    assert list(st) == [0, 4, 4, 4, 4]
    assert np.all(np.isnan(out[:, 1:]))


# ------------------------------------------------------ paper's own values
def test_lox_kinematic_viscosity_table1(orc, species):
    """Table 1: nu_min = 7.7548e-8 m^2/s for the real-gas cases, LOX at
    10 MPa (150 K, Sec. 3.3), Re = u0 L0 / nu = 1547.  Loose (10 %): the
    paper's exact Chung variant and constants are not given."""
    g = GOLDEN["lox_nu_min"]
    out, st = orc.props(species, [g["T"]], [g["p"]], one_hot(1))
    nu = out[4, 0] / out[0, 0]
    assert nu == pytest.approx(g["value"], rel=g["tol_rel"])
    re = GOLDEN["lox_reynolds"]
    assert re["u0"] * re["L0"] / nu == pytest.approx(re["value"], rel=0.1)


@pytest.mark.parametrize("name", ["O2", "CH4"])
def test_pseudo_boiling_shape(orc, species, name):
    """Sec. 2 / Fig. 1: at 10 MPa, pure O2 and CH4 pass smoothly from
    liquid-like to gas-like above Tc: rho(T) decreases monotonically, cp has
    one finite peak."""
    k = W.SPECIES.index(name)
    Tc = GOLDEN["tc_" + name]["value"]
    T = np.linspace(Tc + 2.0, 2.5 * Tc, 600)
    Y = np.zeros((9, T.size))
    Y[k] = 1.0
    out, st = orc.props(species, T, 10e6, Y)
    assert np.all(st == 0)
    assert np.all(np.diff(out[0]) < 0)
    cp = out[3]
    peaks = np.nonzero((cp[1:-1] > cp[:-2]) & (cp[1:-1] > cp[2:]))[0]
    assert len(peaks) == 1
    assert np.isfinite(cp).all()
    assert out[0, 0] / out[0, -1] > 5.0   # large density drop across the line


def test_chung_dilute_conductivity_monatomic_eucken(orc, species):
    """For a monatomic gas (cv = 3/2 R, so Chung's alpha = 0 and Psi = 1)
    the dilute Chung conductivity is the kinetic-theory Eucken value
    lambda = (15/4) R mu / M; 31.2 / R = 3.7525 agrees with 15/4 to 0.07 %."""
    k = W.SPECIES.index("H")
    T = np.array([300.0, 1000.0, 2500.0])
    Y = np.zeros((9, 3))
    Y[k] = 1.0
    _, _, d = orc.diagnose(species, T, np.ones(3), Y)
    M = species.W[k] * 1e-3
    for di in d:
        assert di["cv_ig_molar"] == pytest.approx(1.5 * R, rel=1e-8)
        assert di["lambda_dilute"] == pytest.approx(3.75 * R * di["mu_dilute"] / M, rel=1e-3)


@pytest.mark.parametrize("name", ["O2", "CH4", "CO2", "CO", "H2"])
def test_chung_dilute_conductivity_between_eucken_forms(orc, species, name):
    """Polyatomic non-polar gases: Chung's Psi factor places the dilute
    conductivity between the Eucken (cv + 9/4 R) and modified-Eucken
    (1.32 cv + 1.77 R) values of lambda M / mu, within 8 %."""
    k = W.SPECIES.index(name)
    T = np.array([300.0, 700.0, 1500.0, 2500.0])
    Y = np.zeros((9, T.size))
    Y[k] = 1.0
    _, _, d = orc.diagnose(species, T, np.ones(T.size), Y)
    M = species.W[k] * 1e-3
    for di in d:
        eu = (di["cv_ig_molar"] + 2.25 * R) * di["mu_dilute"] / M
        meu = (1.32 * di["cv_ig_molar"] + 1.77 * R) * di["mu_dilute"] / M
        lo, hi = min(eu, meu), max(eu, meu)
        assert 0.92 * lo <= di["lambda_dilute"] <= 1.08 * hi


# ------------------------------------------------- psi = (d rho / d p)_h
def test_psi_against_constant_enthalpy_differences(orc, species):
    """psi (Sec. 4.1: d rho / d p at constant enthalpy) against central
    differences of rho(p) along constant h, each side through the oracle's own
    T(h, p) inversion: uniform cells, flame-sheet states and pure O2 across
    its pseudo-boiling temperatures at 10 MPa."""
    T, p, Y = W.uniform_cells(300, seed=11)
    Tm, pm, Ym = W.manifold_states(300, seed=12)
    n = 200
    Yo = np.zeros((9, n))
    Yo[W.SPECIES.index("O2")] = 1.0
    T = np.concatenate([T, Tm, np.linspace(140.0, 200.0, n)])
    p = np.concatenate([p, pm, np.full(n, 1e7)])
    Y = np.concatenate([Y, Ym, Yo], axis=1)
    o, st = orc.props_ext(species, T, p, Y)
    dp = 1e-5 * p
    Tp, s1, _ = orc.T_from_h(species, o[2], p + dp, Y, T)
    Tn, s2, _ = orc.T_from_h(species, o[2], p - dp, Y, T)
    rp, _ = orc.props(species, Tp, p + dp, Y)
    rn, _ = orc.props(species, Tn, p - dp, Y)
    ok = (st == 0) & (s1 == 0) & (s2 == 0)
    assert ok.sum() > 750
    fd = (rp[0] - rn[0]) / (2 * dp)
    np.testing.assert_allclose(o[6][ok], fd[ok], rtol=1e-7)


def test_psi_ideal_gas_limit(orc, species):
    """At 1 Pa the gas is ideal: constant h means constant T, so
    psi = rho / p = W / (R T)."""
    T, _, Y = W.uniform_cells(200, seed=13)
    T = 700.0 + (T - 100.0) * (2800.0 / 3400.0)
    p = np.ones(T.size)
    o, st = orc.props_ext(species, T, p, Y)
    assert np.all(st == 0)
    np.testing.assert_allclose(o[6], o[0] / p, rtol=1e-7)
    # the other outputs are those of props; alpha is lambda / cp by definition
    o6, _ = orc.props(species, T, p, Y)
    assert np.array_equal(o[:6], o6)


REF = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fluid_reference_data.json")))


def _cv0_molar(species, k, T):
    """Ideal-gas molar cv of species k at T (NASA-7 low range, T < T_mid)."""
    a = species.nasa_lo[k]
    return R * (a[0] + a[1] * T + a[2] * T ** 2 + a[3] * T ** 3 + a[4] * T ** 4 - 1.0)


def test_chung_polar_terms_against_liquid_water(orc, species):
    """Sec. 2 (Chung's transport model): the polar (mu_r^4) and association
    (kappa) columns of Chung's viscosity coefficients, checked on dense liquid
    water at three measured states (IAPWS-2008 viscosity at the IAPWS-95
    density).  Without water's dipole and association terms the correlation
    is 90-500 % off there; with them, within 5 %."""
    k = W.SPECIES.index("H2O")
    d = REF["water_liquid_viscosity"]
    for s in d["states"]:
        rho_mol = s["rho"] / species.W[k] * 1000.0
        mu, lam, _, _ = orc.chung_pure(species.Tc[k], species.Vc[k], species.omega[k], species.W[k],
                                       species.dipole[k], species.kappa[k], s["T"], rho_mol,
                                       _cv0_molar(species, k, s["T"]))
        assert mu == pytest.approx(s["mu"], rel=d["tol_rel"]), (s, mu)
        mu0, _, _, _ = orc.chung_pure(species.Tc[k], species.Vc[k], species.omega[k], species.W[k], 0.0, 0.0,
                                      s["T"], rho_mol, _cv0_molar(species, k, s["T"]))
        assert abs(mu0 / s["mu"] - 1.0) > 0.5          # the polar terms matter here


def test_chung_dense_terms_against_cryogenic_liquids(orc, species):
    """Sec. 2: the dense-fluid terms of Chung's viscosity (G2 and eta**) and
    conductivity (H2 and the y^2 term), checked on saturated liquid oxygen and
    methane at their normal boiling points (y = rho Vc / 6 near 0.45, where
    these terms carry most of the value)."""
    d = REF["cryogenic_liquids"]
    for s in d["states"]:
        k = W.SPECIES.index(s["species"])
        rho_mol = s["rho"] / species.W[k] * 1000.0
        mu, lam, mu0, lam0 = orc.chung_pure(species.Tc[k], species.Vc[k], species.omega[k], species.W[k],
                                            species.dipole[k], species.kappa[k], s["T"], rho_mol,
                                            _cv0_molar(species, k, s["T"]))
        assert mu == pytest.approx(s["mu"], rel=d["tol_rel"]), (s, mu)
        assert lam == pytest.approx(s["lambda"], rel=d["tol_rel"]), (s, lam)
        assert mu > 5 * mu0 and lam > 5 * lam0            # the dense terms carry the value
