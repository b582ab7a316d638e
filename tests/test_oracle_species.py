"""Pins of the oracle's per-species outputs (Sec. 4.1: standard-state
enthalpies h_k/(R T) and mixture-averaged diffusion coefficients; Sec. 2:
binary diffusion with a high-pressure correction) against closed forms,
kinetic-theory identities and textbook tables, on the CPU."""
import types

import numpy as np
import pytest

from paper_2312_04830_gb300 import workloads as W
from tests.test_oracle_pins import HF298

R = 8.314462618


def one_hot(k, n=1, N=9):
    Y = np.zeros((N, n))
    Y[k] = 1.0
    return Y


def synthetic(W_, Tc, Vc, pc=None):
    """Two or more non-polar species with chosen W [g/mol], Tc [K], Vc
    [cm^3/mol] (NASA data of O2, which the diffusion does not use)."""
    base = W.species_table()
    k = W.SPECIES.index("O2")
    N = len(W_)
    return types.SimpleNamespace(
        W=np.array(W_, float), Tc=np.array(Tc, float), Vc=np.array(Vc, float),
        pc=np.array(pc if pc is not None else [5.0e6] * N, float), omega=np.zeros(N), dipole=np.zeros(N),
        kappa=np.zeros(N), nasa_lo=np.repeat(base.nasa_lo[k:k + 1], N, 0),
        nasa_hi=np.repeat(base.nasa_hi[k:k + 1], N, 0), T_mid=np.full(N, base.T_mid[k]), kij=None)


# --------------------------------------------------------- h_k^0 / (R T)
@pytest.mark.parametrize("name", list(HF298))
def test_hk_RT_formation_enthalpy(orc, species, name):
    """h_k(298.15 K) is the standard enthalpy of formation (JANAF / CODATA)."""
    k = W.SPECIES.index(name)
    hk, _, st = orc.species_props(species, [298.15], [1e5], one_hot(k))
    assert st[0] == 0
    assert hk[k, 0] * R * 298.15 / 1e3 == pytest.approx(HF298[name], abs=0.3)


def test_hk_RT_monatomic_hydrogen_closed_form(orc, species):
    """Atomic H has a constant cp in the data (both sets' a2..a5 terms stay
    below 3e-7 up to 3500 K), so h/(R T) = a1 + a6/T."""
    k = W.SPECIES.index("H")
    for a in (species.nasa_lo[k], species.nasa_hi[k]):
        assert a[0] == pytest.approx(2.5, abs=1e-7)
        assert np.all(np.abs(a[1:5] * 3500.0 ** np.arange(1, 5)) < 3e-7)
    T = np.array([150.0, 300.0, 900.0, 2000.0, 3400.0])
    Y = np.zeros((9, T.size))
    Y[k] = 1.0
    hk, _, _ = orc.species_props(species, T, np.full(T.size, 1e6), Y)
    a = np.where((T < species.T_mid[k])[:, None], species.nasa_lo[k], species.nasa_hi[k])
    assert np.allclose(hk[k], a[:, 0] + a[:, 5] / T, rtol=2e-7, atol=0)


def test_hk_RT_derivative_is_cp(orc, species):
    """d(h_k / R) / dT = cp_k / R: the central difference of T h_k/(R T)
    against each species' ideal-gas cp from the property path (a dropped or
    mis-indexed NASA coefficient fails here)."""
    T = np.array([150.0, 420.0, 800.0, 1600.0, 2900.0])
    dT = 1e-3
    n = T.size
    rng = np.random.default_rng(5)
    Y = W.dirichlet_half(rng, 9, n)
    hp, _, _ = orc.species_props(species, T + dT, np.full(n, 1e6), Y)
    hm, _, _ = orc.species_props(species, T - dT, np.full(n, 1e6), Y)
    fd = ((T + dT) * hp - (T - dT) * hm) / (2 * dT)
    for k in range(9):
        _, _, d = orc.diagnose(species, T, np.full(n, 1.0), one_hot(k, n))
        cpR = np.array([di["cp_ig"] for di in d]) * species.W[k] * 1e-3 / R
        assert np.allclose(fd[k], cpR, rtol=1e-7)


def test_hk_RT_consistent_with_mixture_ideal_enthalpy(orc, species):
    """sum_k Y_k (h_k / R T) R T / W_k is the pinned ideal-gas enthalpy."""
    T, p, Y = W.uniform_cells(200, seed=9)
    hk, _, st = orc.species_props(species, T, p, Y)
    h = (Y * hk / (species.W[:, None] * 1e-3)).sum(0) * R * T
    ref = orc.h_ideal(species, T, Y)
    assert np.all(st == 0)
    assert np.allclose(h, ref, rtol=1e-11, atol=1e-9 * np.abs(ref).max())


# ------------------------------------------------------ collision integral
# Hirschfelder, Curtiss & Bird: Lennard-Jones Omega^(1,1)* (diffusion).
OMEGA11 = {1.0: 1.439, 2.0: 1.075, 5.0: 0.8422, 10.0: 0.7424}


@pytest.mark.parametrize("Ts", list(OMEGA11))
def test_neufeld_diffusion_integral_vs_table(orc, Ts):
    assert orc.neufeld_omega_d(Ts) == pytest.approx(OMEGA11[Ts], rel=2e-3)


# ------------------------------------------------------------ diffusion
@pytest.mark.parametrize("name", ["O2", "CH4", "CO2", "CO", "H2"])
def test_self_diffusion_kinetic_theory_ratio(orc, species, name):
    """Chapman-Enskog: rho D_kk / mu = (6/5) A*, A* = Omega(2,2)*/Omega(1,1)*
    in 1.09..1.12 for T* in 1..10.  The viscosity is the oracle's dilute Chung
    value, whose F_c = 1 - 0.2756 omega factor (non-polar) is divided out."""
    k = W.SPECIES.index(name)
    eps = species.Tc[k] / 1.2593
    T = eps * np.array([1.2, 2.0, 5.0, 9.0])
    T = T[T > 60.0]
    n = T.size
    p = np.full(n, 1e4)
    _, Dk, st = orc.species_props(species, T, p, one_hot(k, n))
    _, _, d = orc.diagnose(species, T, p, one_hot(k, n))
    mu0 = np.array([di["mu_dilute"] for di in d])
    rho = p * species.W[k] * 1e-3 / (R * T)
    Fc = 1.0 - 0.2756 * species.omega[k]
    A = rho * Dk[k] / mu0 * Fc / 1.2
    assert np.all(st == 0)
    assert np.all((A > 1.085) & (A < 1.125)), A


def test_diffusion_inverse_in_pressure(orc, species):
    """Without the high-pressure correction D p depends on T and Y only."""
    T, _, Y = W.uniform_cells(64, seed=3)
    out = []
    for p in (1e5, 1e6, 1e7):
        _, Dk, _ = orc.species_props(species, T, np.full(T.size, p), Y)
        out.append(Dk * p)
    assert np.allclose(out[0], out[1], rtol=1e-14, atol=0)
    assert np.allclose(out[0], out[2], rtol=1e-14, atol=0)


@pytest.mark.parametrize("pair", [("O2", "CH4"), ("H2", "CO2"), ("H2O", "O")])
def test_binary_mixture_ratio_is_molar_mass_ratio(orc, species, pair):
    """Binary A-B: D_Am = D_AB (1 - Y_A)/X_B = D_AB W_B / W_mean, so
    D_Am / D_Bm = W_B / W_A at any composition (mass fractions chosen so
    that Y_A + Y_B = 1 exactly)."""
    a, b = (W.SPECIES.index(s) for s in pair)
    YA = np.array([2.0 ** -30, 0.125, 0.5, 0.875, 1 - 2.0 ** -30])
    n = YA.size
    Y = np.zeros((9, n))
    Y[a], Y[b] = YA, 1 - YA
    T = np.linspace(300.0, 2500.0, n)
    _, Dk, _ = orc.species_props(species, T, np.full(n, 1e6), Y)
    assert np.allclose(Dk[a] / Dk[b], species.W[b] / species.W[a], rtol=1e-12)


def test_diffusion_invariant_to_mass_fraction_scale(orc, species):
    """X_k and the mass share of the other species, sum_{j != k} Y_j / sum Y_j,
    are both invariant to a common factor on Y (inputs whose sum is off 1 by
    less than the accepted 1e-6), so D_k is too; 1 - Y_k would not be."""
    T, p, Y = W.uniform_cells(256, seed=12)
    Y[:, :64] = 0.0
    Y[2, :64], Y[5, :64] = 1 - 2.0 ** -40, 2.0 ** -40     # a species at the edge of purity
    _, D0, _ = orc.species_props(species, T, p, Y)
    _, D1, st = orc.species_props(species, T, p, Y * (1 + 5e-7))
    assert np.all(st == 0)
    assert np.allclose(D1, D0, rtol=2e-14, atol=0)


def test_trace_limits_are_the_binary_coefficient(orc, species):
    """A in trace amount in B and B in trace amount in A both diffuse with the
    one binary D_AB (the pair terms are symmetric)."""
    a, b = W.SPECIES.index("O2"), W.SPECIES.index("H2O")
    Y = np.zeros((9, 2))
    Y[a], Y[b] = [1e-12, 1 - 1e-12], [1 - 1e-12, 1e-12]
    T = np.array([700.0, 700.0])
    _, Dk, _ = orc.species_props(species, T, np.full(2, 1e6), Y)
    assert Dk[a, 0] == pytest.approx(Dk[b, 1], rel=1e-10)


def test_pair_mass_rule(orc):
    """Species equal but for W: D_AB / D_AA = sqrt(W_A / M_AB),
    M_AB = 2 W_A W_B / (W_A + W_B)."""
    WA, WB = 4.0, 44.0
    sp = synthetic([WA, WB], [150.0, 150.0], [90.0, 90.0])
    Y = np.array([[1e-13, 1.0], [1 - 1e-13, 0.0]])
    _, Dk, _ = orc.species_props(sp, [500.0, 500.0], [1e6, 1e6], Y)
    M_AB = 2 * WA * WB / (WA + WB)
    assert Dk[0, 0] / Dk[0, 1] == pytest.approx(np.sqrt(WA / M_AB), rel=1e-11)


def test_pair_size_rule(orc):
    """Species equal but for Vc: sigma_AB is the arithmetic mean, so
    D_AB / D_AA = (sigma_A / sigma_AB)^2 with sigma = 0.809 Vc^(1/3)."""
    VA, VB = 60.0, 250.0
    sp = synthetic([30.0, 30.0], [200.0, 200.0], [VA, VB])
    Y = np.array([[1e-13, 1.0], [1 - 1e-13, 0.0]])
    _, Dk, _ = orc.species_props(sp, [800.0, 800.0], [1e6, 1e6], Y)
    sA, sB = VA ** (1 / 3), VB ** (1 / 3)
    assert Dk[0, 0] / Dk[0, 1] == pytest.approx((sA / (0.5 * (sA + sB))) ** 2, rel=1e-11)


def test_pair_energy_rule(orc):
    """Species equal but for Tc: eps_AB is the geometric mean; at
    T = 2 sqrt(eps_A eps_B) the pair integral is the tabulated Omega(1,1)*(2)."""
    TA, TB = 120.0, 480.0
    sp = synthetic([30.0, 30.0], [TA, TB], [100.0, 100.0])
    eA, eB = TA / 1.2593, TB / 1.2593
    T = 2.0 * np.sqrt(eA * eB)
    Y = np.array([[1e-13, 1.0], [1 - 1e-13, 0.0]])
    _, Dk, _ = orc.species_props(sp, [T, T], [1e6, 1e6], Y)
    ratio = Dk[0, 0] / Dk[0, 1]          # D_AB / D_AA = Omega_D(T/eps_A) / Omega_D(T/eps_AB)
    assert ratio == pytest.approx(orc.neufeld_omega_d(T / eA) / OMEGA11[2.0], rel=2e-3)


def _kay(species, Y, T, p):
    X = Y / species.W[:, None]
    X /= X.sum(0)
    return T / (X * species.Tc[:, None]).sum(0), p / (X * species.pc[:, None]).sum(0)


def test_correction_table_identity_and_constant(orc, species):
    T, p, Y = W.uniform_cells(100, seed=4)
    _, D0, _ = orc.species_props(species, T, p, Y)
    Tr = np.array([0.5, 1.0, 2.0, 8.0])
    pr = np.array([0.1, 1.0, 3.0])
    _, D1, _ = orc.species_props(species, T, p, Y, corr=(Tr, pr, np.ones((4, 3))))
    _, Dc, _ = orc.species_props(species, T, p, Y, corr=(Tr, pr, np.full((4, 3), 0.37)))
    assert np.array_equal(D0, D1)
    assert np.allclose(Dc, 0.37 * D0, rtol=1e-15, atol=0)


def test_correction_table_bilinear_and_clamped(orc, species):
    """A table of f = a + b T_r + c p_r + d T_r p_r (bilinear) on an uneven
    grid is reproduced exactly between its nodes (T_r rows, p_r columns), held
    at its edge value outside, and applied as one factor to every species of
    the cell at the mixture's Kay's-rule pseudo-reduced state."""
    f = lambda x, y: 0.2 + 0.15 * x + 0.05 * y - 0.01 * x * y
    Tr = np.array([0.6, 0.9, 1.05, 1.6, 3.0, 6.0])
    pr = np.array([0.2, 0.8, 1.5, 2.7])
    tab = f(Tr[:, None], pr[None, :])
    T, p, Y = W.uniform_cells(300, seed=6)
    p = p * np.exp(np.random.default_rng(7).uniform(-2.5, 0.4, p.size))
    _, D0, _ = orc.species_props(species, T, p, Y)
    _, D1, _ = orc.species_props(species, T, p, Y, corr=(Tr, pr, tab))
    x, y = _kay(species, Y, T, p)
    expect = f(np.clip(x, Tr[0], Tr[-1]), np.clip(y, pr[0], pr[-1]))
    fac = D1 / D0
    assert np.allclose(fac, expect[None, :], rtol=1e-12, atol=0)
    assert np.any(x > Tr[-1]) and np.any((x > Tr[0]) & (x < Tr[-1]))
    assert np.any(y < pr[0]) and np.any((y > pr[0]) & (y < pr[-1]))


def test_species_bad_input(orc, species):
    T = np.array([300.0, -1.0, 300.0, np.nan])
    Y = np.full((9, 4), 1.0 / 9)
    Y[0, 2] = 0.5
    hk, Dk, st = orc.species_props(species, T, np.full(4, 1e6), Y)
    assert list(st) == [0, 4, 4, 4]
    assert np.all(np.isnan(hk[:, 1:])) and np.all(np.isnan(Dk[:, 1:]))
    assert np.all(np.isfinite(hk[:, 0])) and np.all(Dk[:, 0] > 0)
