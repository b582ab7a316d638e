"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds raw data and random draws only: species constants as published
(critical point, acentric factor, molar mass, Chung's dipole/association inputs,
NASA-7 polynomial coefficients) and the seeded cell-state generators. It holds
none of the method's arithmetic (no mixing, no equation of state, no transport),
so that both sides of every parity test receive identical inputs while sharing
no computation.

Workloads (stand-ins for the paper's 256^3 reacting Taylor-Green-vortex fields,
Table 1 and Sec. 3.3; the paper's CFD data are not available):

* ``uniform_cells``      -- independent cells, T ~ U[100, 3500] K,
  p = 10 MPa x U[0.95, 1.05], Y ~ Dirichlet(0.5) over the 9 species.
* ``flame_vortex_field`` -- a 3-D slab mixture-fraction field distorted by a
  Taylor-Green displacement, with T and Y from a Burke-Schumann LOX/CH4
  flame-sheet profile, p = 10 MPa.
* ``newton_targets``     -- the perturbed temperatures whose enthalpies feed the
  T(h, p, Y) inversion.
* ``training_states``    -- half uniform cells, half flame-sheet states (half of them with noise).
* ``serving_trace``      -- Poisson arrivals of uneven-size client requests.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Species data.  Order fixed: CH4, O2, CO2, H2O, CO, H2, OH, H, O.
#
# Critical constants, acentric factors, critical volumes and dipole moments:
# Poling, Prausnitz & O'Connell, "The Properties of Gases and Liquids", 5th ed.,
# Appendix A.  The radicals OH, H and O have no tabulated critical point; they
# take the parent molecule's (OH <- H2O, H <- H2, O <- O2) critical constants
# with dipole and association set to zero, and keep their own molar mass and
# NASA-7 data.  Association factor of water (0.076): Chung et al. (1988).
#
# NASA-7 two-range coefficients: the GRI-Mech 3.0 thermodynamic data set
# (200-1000 K low range, 1000-3500 K high range).  Each set is given as
# (a1..a7).  The tests check each set for continuity of cp, h and s at T_mid
# and for the standard enthalpy of formation at 298.15 K.
# ---------------------------------------------------------------------------

SPECIES = ("CH4", "O2", "CO2", "H2O", "CO", "H2", "OH", "H", "O")

# atoms of carbon, hydrogen and oxygen per molecule (Bilger's mixture fraction)
ATOMS_CHO = ((1, 4, 0), (0, 0, 2), (1, 0, 2), (0, 2, 1), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 1, 0), (0, 0, 1))
# the two streams of the flame-vortex field: pure CH4 fuel, pure O2 oxidiser
Y_FUEL = (1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0)
Y_OX = (0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0)

# molar mass [g/mol]
W_G_PER_MOL = (16.043, 31.998, 44.009, 18.015, 28.010, 2.016, 17.007, 1.008, 15.999)
# critical temperature [K]
TC_K = (190.56, 154.58, 304.12, 647.14, 132.85, 32.98, 647.14, 32.98, 154.58)
# critical pressure [Pa]
PC_PA = (4.599e6, 5.043e6, 7.374e6, 22.064e6, 3.494e6, 1.293e6, 22.064e6, 1.293e6, 5.043e6)
# acentric factor [-]
OMEGA = (0.011, 0.022, 0.225, 0.344, 0.045, -0.217, 0.344, -0.217, 0.022)
# critical molar volume [cm^3/mol]
VC_CM3_PER_MOL = (98.6, 73.37, 94.07, 55.95, 93.10, 64.20, 55.95, 64.20, 73.37)
# dipole moment [debye]
DIPOLE_DEBYE = (0.0, 0.0, 0.0, 1.8, 0.1, 0.0, 0.0, 0.0, 0.0)
# Chung association factor kappa [-]
KAPPA_ASSOC = (0.0, 0.0, 0.0, 0.076, 0.0, 0.0, 0.0, 0.0, 0.0)

NASA_T_LOW = (200.0,) * 9
NASA_T_MID = (1000.0,) * 9
NASA_T_HIGH = (3500.0,) * 9

# (low-range a1..a7, high-range a1..a7)
NASA7 = {
    "CH4": ((5.14987613e+00, -1.36709788e-02, 4.91800599e-05, -4.84743026e-08, 1.66693956e-11,
             -1.02466476e+04, -4.64130376e+00),
            (7.48514950e-02, 1.33909467e-02, -5.73285809e-06, 1.22292535e-09, -1.01815230e-13,
             -9.46834459e+03, 1.84373180e+01)),
    "O2": ((3.78245636e+00, -2.99673416e-03, 9.84730201e-06, -9.68129509e-09, 3.24372837e-12,
            -1.06394356e+03, 3.65767573e+00),
           (3.28253784e+00, 1.48308754e-03, -7.57966669e-07, 2.09470555e-10, -2.16717794e-14,
            -1.08845772e+03, 5.45323129e+00)),
    "CO2": ((2.35677352e+00, 8.98459677e-03, -7.12356269e-06, 2.45919022e-09, -1.43699548e-13,
             -4.83719697e+04, 9.90105222e+00),
            (3.85746029e+00, 4.41437026e-03, -2.21481404e-06, 5.23490188e-10, -4.72084164e-14,
             -4.87591660e+04, 2.27163806e+00)),
    "H2O": ((4.19864056e+00, -2.03643410e-03, 6.52040211e-06, -5.48797062e-09, 1.77197817e-12,
             -3.02937267e+04, -8.49032208e-01),
            (3.03399249e+00, 2.17691804e-03, -1.64072518e-07, -9.70419870e-11, 1.68200992e-14,
             -3.00042971e+04, 4.96677010e+00)),
    "CO": ((3.57953347e+00, -6.10353680e-04, 1.01681433e-06, 9.07005884e-10, -9.04424499e-13,
            -1.43440860e+04, 3.50840928e+00),
           (2.71518561e+00, 2.06252743e-03, -9.98825771e-07, 2.30053008e-10, -2.03647716e-14,
            -1.41518724e+04, 7.81868772e+00)),
    "H2": ((2.34433112e+00, 7.98052075e-03, -1.94781510e-05, 2.01572094e-08, -7.37611761e-12,
            -9.17935173e+02, 6.83010238e-01),
           (3.33727920e+00, -4.94024731e-05, 4.99456778e-07, -1.79566394e-10, 2.00255376e-14,
            -9.50158922e+02, -3.20502331e+00)),
    "OH": ((3.99201543e+00, -2.40131752e-03, 4.61793841e-06, -3.88113333e-09, 1.36411470e-12,
            3.61508056e+03, -1.03925458e-01),
           (3.09288767e+00, 5.48429716e-04, 1.26505228e-07, -8.79461556e-11, 1.17412376e-14,
            3.85865700e+03, 4.47669610e+00)),
    "H": ((2.50000000e+00, 7.05332819e-13, -1.99591964e-15, 2.30081632e-18, -9.27732332e-22,
           2.54736599e+04, -4.46682853e-01),
          (2.50000001e+00, -2.30842973e-11, 1.61561948e-14, -4.73515235e-18, 4.98197357e-22,
           2.54736599e+04, -4.46682914e-01)),
    "O": ((3.16826710e+00, -3.27931884e-03, 6.64306396e-06, -6.12806624e-09, 2.11265971e-12,
           2.91222592e+04, 2.05193346e+00),
          (2.56942078e+00, -8.59741137e-05, 4.19484589e-08, -1.00177799e-11, 1.22833691e-15,
           2.92175791e+04, 4.78433864e+00)),
}


class SpeciesTable:
    """Plain arrays of the species data above (SI except where noted).

    Fields: ``W`` [g/mol], ``Tc`` [K], ``pc`` [Pa], ``omega`` [-],
    ``Vc`` [cm^3/mol], ``dipole`` [debye], ``kappa`` [-],
    ``nasa_lo`` / ``nasa_hi`` [N, 7], ``T_low`` / ``T_mid`` / ``T_high`` [K],
    ``kij`` [N, N] binary interaction parameters (zeros by default).
    """

    def __init__(self, names=SPECIES, kij=None):
        idx = [SPECIES.index(s) for s in names]
        self.names = tuple(names)
        self.n = len(idx)
        pick = lambda seq: np.array([seq[i] for i in idx], dtype=np.float64)
        self.W = pick(W_G_PER_MOL)
        self.Tc = pick(TC_K)
        self.pc = pick(PC_PA)
        self.omega = pick(OMEGA)
        self.Vc = pick(VC_CM3_PER_MOL)
        self.dipole = pick(DIPOLE_DEBYE)
        self.kappa = pick(KAPPA_ASSOC)
        self.T_low = pick(NASA_T_LOW)
        self.T_mid = pick(NASA_T_MID)
        self.T_high = pick(NASA_T_HIGH)
        self.nasa_lo = np.array([NASA7[SPECIES[i]][0] for i in idx], dtype=np.float64)
        self.nasa_hi = np.array([NASA7[SPECIES[i]][1] for i in idx], dtype=np.float64)
        self.kij = (np.zeros((self.n, self.n)) if kij is None
                    else np.ascontiguousarray(kij, dtype=np.float64))

    def subset(self, names):
        return SpeciesTable(names)


def species_table(kij=None) -> SpeciesTable:
    return SpeciesTable(SPECIES, kij=kij)


# ---------------------------------------------------------------------------
# Cell-state generators.  Every generator returns SoA float64 arrays:
# T [n], p [n], Y [N, n] (species-major, Y[k, i]).
# ---------------------------------------------------------------------------

P_REF = 10.0e6  # operating pressure of the paper's cases [Pa] (Sec. 3)


def dirichlet_half(rng, k: int, n: int) -> np.ndarray:
    """[k, n] draws of Dirichlet(0.5 * 1_k).  Gamma(1/2) is half a squared
    standard normal, so normalised squared normals are exact Dirichlet(1/2)
    draws (and much faster than rejection-sampled gammas)."""
    z = rng.standard_normal((k, n))
    z *= z
    z /= z.sum(axis=0, keepdims=True)
    return z


def uniform_cells(n: int = 32768, seed: int = 20231204):
    """Independent cells: T ~ U[100, 3500] K, p = 10 MPa x U[0.95, 1.05],
    Y ~ Dirichlet(0.5 * 1_9).  Draw order: T, p, Y (PCG64)."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(100.0, 3500.0, n)
    p = P_REF * rng.uniform(0.95, 1.05, n)
    Y = dirichlet_half(rng, len(SPECIES), n)
    return T, p, np.ascontiguousarray(Y)


# Burke-Schumann flame-sheet constants (LOX/CH4; the paper's oxidiser is at
# 150 K, Sec. 3.3; the synthetic field uses 120 K)
T_OX = 120.0
T_FUEL = 300.0
T_ST = 3500.0


def _stoich():
    w = dict(zip(SPECIES, W_G_PER_MOL))
    s = 2.0 * w["O2"] / w["CH4"]                   # oxidiser-to-fuel mass ratio
    z_st = 1.0 / (1.0 + s)
    f_co2 = w["CO2"] / (w["CO2"] + 2.0 * w["H2O"])  # CO2 share of product mass
    return z_st, f_co2


def flame_sheet_state(Zmix: np.ndarray):
    """T and Y of a Burke-Schumann CH4/O2 flame sheet at mixture fraction Z."""
    z_st, f_co2 = _stoich()
    Zmix = np.asarray(Zmix, dtype=np.float64)
    lean = Zmix <= z_st
    n = Zmix.size
    Y = np.zeros((len(SPECIES), n))
    yp = np.where(lean, Zmix / z_st, (1.0 - Zmix) / (1.0 - z_st))
    Y[SPECIES.index("O2")] = np.where(lean, 1.0 - Zmix / z_st, 0.0)
    Y[SPECIES.index("CH4")] = np.where(lean, 0.0, (Zmix - z_st) / (1.0 - z_st))
    Y[SPECIES.index("CO2")] = f_co2 * yp
    Y[SPECIES.index("H2O")] = (1.0 - f_co2) * yp
    T = np.where(lean, T_OX + (T_ST - T_OX) * Zmix / z_st,
                 T_FUEL + (T_ST - T_FUEL) * (1.0 - Zmix) / (1.0 - z_st))
    return T, Y


def flame_vortex_field(g: int = 256, L: float = 1.0, amp: float = 0.3, delta_frac: float = 1.0 / 40.0,
                       p: float = P_REF, z_range=None):
    """Flame-vortex field on a g^3 grid of [0, L]^3, cell-major order i = (ix*g + iy)*g + iz.

    Mixture fraction Z = 0.5 (1 + tanh(x'/delta)) with x' = (x - L/2) +
    amp*L*cos(2 pi y/L) cos(2 pi z/L), delta = delta_frac*L; Z -> 1 on the fuel
    side.  T, Y from ``flame_sheet_state``; p uniform but stored per cell.
    ``z_range`` = (ix0, ix1) generates only slabs ix0 <= ix < ix1.
    """
    ix0, ix1 = (0, g) if z_range is None else z_range
    c = (np.arange(g, dtype=np.float64) + 0.5) * (L / g)
    x = c[ix0:ix1][:, None, None]
    y = c[None, :, None]
    z = c[None, None, :]
    xp = (x - 0.5 * L) + amp * L * np.cos(2.0 * np.pi * y / L) * np.cos(2.0 * np.pi * z / L)
    Zmix = 0.5 * (1.0 + np.tanh(xp / (delta_frac * L)))
    Zmix = np.ascontiguousarray(Zmix).reshape(-1)
    T, Y = flame_sheet_state(Zmix)
    P = np.full(Zmix.size, p)
    return T, P, np.ascontiguousarray(Y)


def newton_targets(T: np.ndarray, seed: int = 20231205, rel: float = 0.05,
                   lo: float = 100.0, hi: float = 3500.0):
    """Perturbed temperatures T_true = clip(T (1 + U[-rel, rel]), lo, hi).

    The inversion workload evaluates h* = h(T_true, p, Y) and starts the
    Newton iteration from the unperturbed T."""
    rng = np.random.default_rng(seed)
    return np.clip(T * (1.0 + rng.uniform(-rel, rel, T.size)), lo, hi)


def manifold_states(n: int, seed: int, p_jitter: bool = True, exact_frac: float = 0.5):
    """Flame-sheet states with noise: Z ~ U[0,1] for half of the states and
    Z = (1 + tanh s) / 2 with s ~ U[-5, 5] for the other half (the mixture
    fractions of a thin flame, piled up at the pure-oxidiser and pure-fuel
    ends as in the flame-vortex field); T (1 + N(0, 0.03));
    Y <- normalise(Y + 0.02 Dirichlet(0.5)) for a fraction 1 - exact_frac of
    the states, the flame-sheet composition itself for the others (fields of
    flame sheets have exact zeros in Y, a corner of the simplex that noisy
    compositions do not reach); p = 10 MPa x U[0.95, 1.05]."""
    rng = np.random.default_rng(seed)
    Zmix = rng.uniform(0.0, 1.0, n)
    thin = rng.uniform(0.0, 1.0, n) < 0.5
    Zmix[thin] = 0.5 * (1.0 + np.tanh(rng.uniform(-5.0, 5.0, int(thin.sum()))))
    T, Y = flame_sheet_state(Zmix)
    T = T * (1.0 + rng.normal(0.0, 0.03, n))
    T = np.clip(T, 100.0, 3500.0)
    noisy = rng.uniform(0.0, 1.0, n) >= exact_frac
    Y = Y + 0.02 * dirichlet_half(rng, len(SPECIES), n) * noisy
    Y /= Y.sum(axis=0, keepdims=True)
    p = P_REF * (rng.uniform(0.95, 1.05, n) if p_jitter else np.ones(n))
    return T, p, np.ascontiguousarray(Y)


def training_states(n: int, seed: int = 20231207):
    """Half uniform cells (as ``uniform_cells``), half flame-sheet states (as
    ``manifold_states``: half of them with noisy compositions)."""
    n_u = n // 2
    Tu, pu, Yu = uniform_cells(n_u, seed)
    Tm, pm, Ym = manifold_states(n - n_u, seed + 1000003)
    return (np.concatenate([Tu, Tm]), np.concatenate([pu, pm]),
            np.ascontiguousarray(np.concatenate([Yu, Ym], axis=1)))


def augmented_field_states(n: int, seed: int, grid: int = 64, a2: float = 20.0):
    """The paper's data augmentation (Sec. 4.2, its equation for t): new states
    t = c + a1 (max(h) - min(h)) / a2 around samples c of a flow field, for
    every variable h, with a1 ~ U[-1, 1] drawn per state and variable and a2 a
    fixed divisor.  The samples c are cells of the flame-vortex field (the
    stand-in for the paper's first TGV time steps); T is clipped to
    [100, 3500] K, mass fractions to [0, 1] and renormalised (the paper's
    constraint that mixture fractions stay in [0, 1]); the positivity of the
    density is left to the labelling filter.  p, uniform in the field, has no
    range and so stays at the field's value."""
    rng = np.random.default_rng(seed)
    Tc, pc, Yc = flame_vortex_field(grid)
    pick = rng.integers(0, Tc.size, n)
    T, p, Y = Tc[pick], pc[pick], Yc[:, pick]
    span = lambda v, axis=None: v.max(axis=axis) - v.min(axis=axis)
    T = np.clip(T + rng.uniform(-1.0, 1.0, n) * span(Tc) / a2, 100.0, 3500.0)
    p = p + rng.uniform(-1.0, 1.0, n) * span(pc) / a2
    Y = Y + rng.uniform(-1.0, 1.0, Y.shape) * (span(Yc, axis=1) / a2)[:, None]
    Y = np.clip(Y, 0.0, 1.0)
    Y /= Y.sum(axis=0, keepdims=True)
    return T, p, np.ascontiguousarray(Y)


def serving_trace(n_clients: int = 64, per_client: int = 16, seed: int = 20231206,
                  g_lo: int = 32, g_hi: int = 256, frac_props: float = 0.7):
    """Request trace: per request a grid edge g = round(exp(U[ln g_lo, ln g_hi])),
    a kind (0 = forward properties with prob. ``frac_props``, 1 = T from h) and a
    client id.  Arrival times are drawn separately (``poisson_arrivals``) once
    the single-stream service rate is known."""
    rng = np.random.default_rng(seed)
    m = n_clients * per_client
    g = np.rint(np.exp(rng.uniform(np.log(g_lo), np.log(g_hi), m))).astype(np.int64)
    kind = (rng.uniform(0.0, 1.0, m) >= frac_props).astype(np.int32)
    client = np.repeat(np.arange(n_clients), per_client)
    order = rng.permutation(m)
    return g[order], kind[order], client[order]


def poisson_arrivals(m: int, rate_per_s: float, seed: int = 20231208):
    """Cumulative arrival times [s] of m requests at an aggregate Poisson rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, m))
