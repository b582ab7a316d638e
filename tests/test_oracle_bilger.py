"""Pins of the oracle's Bilger mixture fraction (the composition input of the
paper's networks, Sec. 4.1) on the CPU: the streams, the flame sheet it
parametrises, element conservation and linearity."""
import numpy as np

from paper_2312_04830_gb300 import workloads as W


def z_of(orc, species, Y):
    return orc.bilger_z(species, W.ATOMS_CHO, W.Y_FUEL, W.Y_OX, Y)


def test_streams_are_zero_and_one(orc, species):
    Y = np.array([W.Y_OX, W.Y_FUEL]).T
    assert list(z_of(orc, species, Y)) == [0.0, 1.0]


def test_flame_sheet_states_return_their_mixture_fraction(orc, species):
    """A Burke-Schumann state at mixture fraction Z holds the elements of the
    unburnt mix Z fuel + (1 - Z) oxidiser, so Bilger's Z of it is Z, lean and
    rich side alike (a wrong coupling coefficient breaks this on the burnt
    side)."""
    Z = np.linspace(0.0, 1.0, 1001)
    _, Y = W.flame_sheet_state(Z)
    assert np.allclose(z_of(orc, species, Y), Z, rtol=0, atol=2e-15)


def test_element_conserving_reactions_leave_z_unchanged(orc, species):
    """Moving mass along any stoichiometric reaction (CH4 oxidation, H2 and
    CO oxidation, dissociations) keeps every element and so Z."""
    idx = {s: i for i, s in enumerate(W.SPECIES)}
    reactions = [{"CH4": -1, "O2": -2, "CO2": 1, "H2O": 2}, {"H2": -2, "O2": -1, "H2O": 2},
                 {"CO": -2, "O2": -1, "CO2": 2}, {"H2": -1, "H": 2}, {"O2": -1, "O": 2},
                 {"H": -1, "O": -1, "OH": 1}, {"H2O": -1, "H": -1, "OH": 1, "H2": 1}]
    rng = np.random.default_rng(3)
    Y0 = W.dirichlet_half(rng, 9, 400)
    Z0 = z_of(orc, species, Y0)
    Y = Y0.copy()
    for r in reactions:
        nu = np.zeros(9)
        for s, v in r.items():
            nu[idx[s]] = v * species.W[idx[s]]          # mass change per unit extent
        assert abs(nu.sum()) < 1e-9 * np.abs(nu).sum()  # the reaction conserves mass
        # largest extent that keeps every mass fraction non-negative, then a random share of it
        lim = np.min(np.where(nu[:, None] < 0, Y / -np.minimum(nu[:, None], -1e-300), np.inf), axis=0)
        Y = Y + nu[:, None] * (rng.uniform(0.0, 1.0, Y.shape[1]) * lim)[None, :]
        Y = np.maximum(Y, 0.0)
    assert np.abs(Y - Y0).max() > 0.05
    assert np.allclose(z_of(orc, species, Y), Z0, rtol=0, atol=1e-12)


def test_linear_in_composition(orc, species):
    rng = np.random.default_rng(4)
    Y1, Y2 = W.dirichlet_half(rng, 9, 100), W.dirichlet_half(rng, 9, 100)
    a = rng.uniform(0.0, 1.0, 100)
    Zm = z_of(orc, species, a * Y1 + (1 - a) * Y2)
    assert np.allclose(Zm, a * z_of(orc, species, Y1) + (1 - a) * z_of(orc, species, Y2), rtol=0, atol=1e-13)


def test_hydrogen_rich_cells_leave_the_unit_interval(orc, species):
    """Z only spans [0, 1] on mixtures of the two streams: pure H2 carries more
    of the fuel's coupling function than CH4 itself."""
    Y = np.zeros((9, 1))
    Y[W.SPECIES.index("H2")] = 1.0
    assert z_of(orc, species, Y)[0] > 1.5
