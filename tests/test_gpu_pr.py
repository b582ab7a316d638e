"""Parity of the CUDA property path with the FP64 oracle (GPU).

Every call goes through the C ABI (ctypes binding).  Inputs come from the
seeded generators; expected values come from the oracle only.
"""
import numpy as np
import pytest

from paper_2312_04830_gb300 import workloads as W

from .parity import assert_fp64_parity, cond_numbers, error_summary, root_sensitivity_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(prlib, cuda, species):
    from paper_2312_04830_gb300 import binding
    c = binding.PropertyContext(species)
    yield c
    c.close()


def to_dev(a, dtype, cuda):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=cuda)


def run_props(ctx, T, p, Y, cuda, precision="fp64"):
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    out, st = ctx.props(to_dev(T, dt, cuda), to_dev(p, dt, cuda), to_dev(Y, dt, cuda), precision=precision)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), st.cpu().numpy()


def oracle_props(orc, species, T, p, Y, **kw):
    out, st, d = orc.diagnose(species, T, p, Y, **kw)
    return out, st, cond_numbers(d)


def check(orc, species, g, gs, T, p, Y, label, expect_ill=False, expect_ambiguous=False, **kw):
    """FP64 parity by the rule of tests/parity.py, the allowances computed by
    the oracle (Chung cancellation ratios, outputs at a moved root)."""
    o, os_, d = orc.diagnose(species, T, p, Y, **kw)
    tb = orc.Table(species, **kw)
    zs = lambda idx, Z, dz, oo: root_sensitivity_bound(orc, tb, T, p, Y, idx, Z, dz, oo)
    return assert_fp64_parity(g, gs, o, os_, T, d, label=label, zsens=zs, expect_ill=expect_ill,
                              expect_ambiguous=expect_ambiguous)


# ------------------------------------------------------------------ FP64
def test_props_fp64_uniform_cells(ctx, orc, species, cuda):
    """32^3 independent cells: T ~ U[100, 3500] K, p = 10 MPa +-5 %, Dirichlet Y."""
    T, p, Y = W.uniform_cells(32768)
    g, gs = run_props(ctx, T, p, Y, cuda)
    rep = check(orc, species, g, gs, T, p, Y, "uniform")
    assert rep["n_ok"] > 32000


@pytest.mark.parametrize("n", [1, 31, 127, 128, 129, 1000, 4099])
def test_props_fp64_ragged_sizes(ctx, orc, species, cuda, n):
    T, p, Y = W.uniform_cells(n, seed=100 + n)
    g, gs = run_props(ctx, T, p, Y, cuda)
    check(orc, species, g, gs, T, p, Y, f"n={n}")


def test_props_empty_is_noop(ctx, cuda):
    import torch
    z = torch.empty(0, dtype=torch.float64, device=cuda)
    out, st = ctx.props(z, z, torch.empty((9, 0), dtype=torch.float64, device=cuda))
    assert out.shape == (6, 0)


def _edge_states(species):
    Ts, ps, Ys = [], [], []
    def add(T, p, k=None, Y=None):
        y = np.zeros(9)
        if k is not None:
            y[k] = 1.0
        else:
            y[:] = Y
        Ts.append(T); ps.append(p); Ys.append(y)
    for k in range(9):
        add(species.Tc[k], species.pc[k], k)                         # critical point (ill-conditioned)
        add(species.Tc[k] * 1.001, species.pc[k] * 1.01, k)
        add(1500.0, 1.0, k)                                          # ideal-gas limit
        add(3500.0, 10.5e6, k)
    for name in ("H2O", "CO2"):                                      # subcritical: two physical roots
        k = W.SPECIES.index(name)
        for tr in np.linspace(0.55, 0.98, 12):
            for pr in np.linspace(0.05, 0.9, 12):
                add(tr * species.Tc[k], pr * species.pc[k], k)
    zm = np.linspace(0, 1, 41)                                       # flame sheet (LOX at 120 K, CH4 at 300 K)
    Tf, Yf = W.flame_sheet_state(zm)
    for i in range(zm.size):
        add(Tf[i], 10e6, Y=Yf[:, i])
    # degenerate inputs: status 4 expected
    add(-5.0, 10e6, 1); add(np.nan, 10e6, 1); add(300.0, 0.0, 1); add(300.0, np.inf, 1)
    y = np.zeros(9); y[1] = 0.9; add(300.0, 10e6, Y=y)              # sum Y = 0.9
    y = np.zeros(9); y[1] = 1.1; y[2] = -0.1; add(300.0, 10e6, Y=y)  # negative Y
    return np.array(Ts), np.array(ps), np.array(Ys).T.copy()


def test_props_fp64_edge_cases(ctx, orc, species, cuda):
    T, p, Y = _edge_states(species)
    g, gs = run_props(ctx, T, p, Y, cuda)
    rep = check(orc, species, g, gs, T, p, Y, "edge", expect_ill=True, expect_ambiguous=True)
    o, os_, cond = oracle_props(orc, species, T, p, Y)
    assert rep["n_ill"] + rep["n_ambiguous"] >= 6     # the critical points
    assert np.count_nonzero(os_ == 4) == 6
    assert np.all(gs[os_ == 4] == 4)


def test_props_fp64_kij(prlib, orc, cuda):
    """Non-zero symmetric k_ij: the O(N^2) mixing path."""
    from paper_2312_04830_gb300 import binding
    rng = np.random.default_rng(5)
    k = rng.uniform(-0.05, 0.15, (9, 9))
    k = 0.5 * (k + k.T)
    np.fill_diagonal(k, 0.0)
    sp = W.species_table(kij=k)
    c = binding.PropertyContext(sp)
    T, p, Y = W.uniform_cells(8192, seed=41)
    g, gs = run_props(c, T, p, Y, cuda)
    check(orc, sp, g, gs, T, p, Y, "kij")
    c.close()


@pytest.mark.parametrize("names", [("O2",), ("CH4", "O2"), tuple(W.SPECIES) + ("O2",),
                                   tuple(W.SPECIES) + ("CH4", "CO2", "H2O", "H2", "CO", "O2", "O", "H")])
def test_props_fp64_species_counts(prlib, orc, cuda, names):
    """1, 2, 10 and 17 species (the 17 a RAMEC-sized table), padded kernels."""
    from paper_2312_04830_gb300 import binding
    sp = W.SpeciesTable(names)
    c = binding.PropertyContext(sp)
    rng = np.random.default_rng(len(names))
    n = 3000
    T = rng.uniform(100, 3500, n)
    p = 1e7 * rng.uniform(0.95, 1.05, n)
    Y = rng.dirichlet(np.full(len(names), 0.5), n).T.copy()
    g, gs = run_props(c, T, p, Y, cuda)
    check(orc, sp, g, gs, T, p, Y, f"N={len(names)}")
    c.close()


def test_props_fp64_transport_xavg_and_printed(prlib, orc, species, cuda):
    from paper_2312_04830_gb300 import binding
    T, p, Y = W.uniform_cells(4096, seed=61)
    for kw in ({"transport_xavg": True}, {"printed_constants": True}):
        c = binding.PropertyContext(species, **kw)
        g, gs = run_props(c, T, p, Y, cuda)
        okw = {"transport_rule": 1} if "transport_xavg" in kw else {"printed_constants": True}
        check(orc, species, g, gs, T, p, Y, str(kw), **okw)
        c.close()


def test_props_strided_Y_and_output_subsets(ctx, orc, species, cuda):
    """Y as a slice of a wider array (ldY > n); skipping mu/lambda leaves the
    thermodynamic outputs bit-identical."""
    import torch
    T, p, Y = W.uniform_cells(5000, seed=71)
    Ywide = np.zeros((9, 6000))
    Ywide[:, :5000] = Y
    Yd = torch.as_tensor(Ywide, device=cuda)[:, :5000]
    Td, pd = torch.as_tensor(T, device=cuda), torch.as_tensor(p, device=cuda)
    full, st = ctx.props(Td, pd, Yd)
    thermo, st2 = ctx.props(Td, pd, Yd, outputs=("rho", "Z", "h", "cp"))
    torch.cuda.synchronize()
    assert torch.equal(full[:4], thermo[:4])
    check(orc, species, full.cpu().numpy(), st.cpu().numpy(), T, p, Y, "strided")


def test_props_deterministic(ctx, cuda):
    import torch
    T, p, Y = W.uniform_cells(20000, seed=81)
    a, _ = run_props(ctx, T, p, Y, cuda)
    b, _ = run_props(ctx, T, p, Y, cuda)
    assert np.array_equal(a, b, equal_nan=True)


# ---------------------------------------------------------------- Newton
def test_T_from_h_fp64(ctx, orc, species, cuda):
    """T(h*, p, Y) on the uniform cells: h* = h_oracle(T_true), start from a
    guess within +-5 %; the GPU's T equals the oracle's inversion."""
    T, p, Y = W.uniform_cells(32768, seed=91)
    Ttrue = W.newton_targets(T, seed=92)
    hs, sts = orc.props(species, Ttrue, p, Y)
    hstar = hs[2]
    To, sto, ito = orc.T_from_h(species, hstar, p, Y, T)
    import torch
    Tg, stg, itg = ctx.T_from_h(to_dev(hstar, torch.float64, cuda), to_dev(p, torch.float64, cuda),
                                to_dev(Y, torch.float64, cuda), to_dev(T, torch.float64, cuda))
    Tg, stg, itg = Tg.cpu().numpy(), stg.cpu().numpy(), itg.cpu().numpy()
    ok = (sto == 0) & (sts == 0)
    assert ok.sum() > 32000
    assert np.all(stg[ok] == 0)
    np.testing.assert_allclose(Tg[ok], To[ok], rtol=1e-10)
    np.testing.assert_allclose(Tg[ok], Ttrue[ok], rtol=1e-10)
    assert itg[ok].max() <= 60


def test_T_from_h_status_codes(ctx, orc, species, cuda):
    import torch
    n = 6
    Y = np.zeros((9, n)); Y[0] = 1.0
    p = np.full(n, 10e6)
    hstar = np.array([-1e9, 1e9, np.nan, 0.0, 1e5, -4e6])
    Tg = np.array([300.0, 300.0, 300.0, 1e4, 1.0, 500.0])
    To, sto, _ = orc.T_from_h(species, hstar, p, Y, Tg)
    d = lambda a: to_dev(a, torch.float64, cuda)
    T2, st2, _ = ctx.T_from_h(d(hstar), d(p), d(Y), d(Tg))
    T2, st2 = T2.cpu().numpy(), st2.cpu().numpy()
    assert list(st2) == list(sto)
    okm = sto != 4
    np.testing.assert_allclose(T2[okm], To[okm], rtol=1e-10)


# ------------------------------------------------------ reduced precision
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_reduced_precision_error_budget(ctx, orc, species, cuda, precision):
    """FP32 and mixed paths: error distribution against the FP64 oracle on
    inputs rounded to FP32 (the oracle sees the same rounded inputs)."""
    T, p, Y = W.uniform_cells(32768, seed=101)
    T32, p32 = T.astype(np.float32).astype(np.float64), p.astype(np.float32).astype(np.float64)
    Y32 = Y.astype(np.float32).astype(np.float64)
    g, gs = run_props(ctx, T32, p32, Y32, cuda, precision=precision)
    o, os_, cond = oracle_props(orc, species, T32, p32, Y32)
    m = (os_ == 0) & (gs == 0) & (cond < 1e4)
    assert m.sum() > 32000
    summ = error_summary(g, o, T32, m)
    print(precision, summ)
    for name, s in summ.items():
        assert s["median"] < 1e-5, (name, s)
        assert s["p99"] < 1e-3, (name, s)


def test_fp64_inversion_one_step_acceptance(ctx, orc, species, cuda):
    """The FP64 inversion takes the first FP64 Newton step after the FP32
    warm start without a second evaluation only on smooth single-root states
    away from the pseudo-boiling band and from the kinks of h(T): on O2 and
    CH4 across their pseudo-boiling temperatures at 10 MPa, on cells next to
    the NASA-7 range switch (1000 K) and on ordinary uniform cells, T equals
    the oracle's inversion and the true T to 1e-10 (within 0.1 mK of the
    range switch, where the fits' small step in h gives h(T) = h* two roots,
    the GPU's T solves h(T) = h* to 1e-12); band cells (cp > 3.3 x the
    ideal-gas cp) and cells within 5 mK of 1000 K take two or more FP64
    evaluations, and most ordinary cells take one."""
    import torch
    rng = np.random.default_rng(37)
    n = 6144
    k_o2, k_ch4 = W.SPECIES.index("O2"), W.SPECIES.index("CH4")
    Y = np.zeros((9, n))
    T = np.empty(n)
    Y[k_o2, :2048] = 1.0
    T[:2048] = rng.uniform(140.0, 200.0, 2048)                 # O2 across its pseudo-boiling band
    Y[k_ch4, 2048:4096] = 1.0
    T[2048:4096] = rng.uniform(190.0, 280.0, 2048)             # CH4
    Tu, pu, Yu = W.uniform_cells(2048, seed=38)                 # ordinary cells, a few at the range switch
    T[4096:], Y[:, 4096:] = Tu, Yu
    T[4096:4352] = 1000.0 + rng.uniform(-0.005, 0.005, 256)
    p = np.full(n, 10e6)
    p[4096:] = pu
    hs, sts = orc.props(species, T, p, Y)
    guess = T * (1 + rng.uniform(-0.05, 0.05, n))
    To, sto, _ = orc.T_from_h(species, hs[2], p, Y, guess)
    d64 = lambda a: to_dev(a, torch.float64, cuda)
    Tg, stg, itg = ctx.T_from_h(d64(hs[2]), d64(p), d64(Y), d64(guess))
    Tg, stg, itg = Tg.cpu().numpy(), stg.cpu().numpy(), itg.cpu().numpy()
    ok = (sto == 0) & (sts == 0)
    assert ok.sum() > 6000
    assert np.all(stg[ok] == 0)
    # the NASA-7 fits do not meet exactly at their range switch: h(T) drops by
    # ~0.01 J/kg across 1000 K here, so h(T) = h* has a root on either side
    # within ~1e-5 K of it; there the GPU's T must solve h(T) = h*, whichever
    # root it found, and elsewhere it must equal the oracle's root
    near = np.abs(T - 1000.0) < 1e-4
    far = ok & ~near
    np.testing.assert_allclose(Tg[far], To[far], rtol=1e-10)
    np.testing.assert_allclose(Tg[far], T[far], rtol=1e-10)
    hn, stn = orc.props(species, Tg[ok & near], p[ok & near], Y[:, ok & near])
    assert np.all(stn == 0)
    assert np.all(np.abs(hn[2] - hs[2][ok & near]) <= 1e-12 * np.abs(hs[2][ok & near]))
    cp = hs[3]
    dT = 1e-3 * T
    ratio = cp / ((orc.h_ideal(species, T + dT, Y) - orc.h_ideal(species, T - dT, Y)) / (2 * dT))
    band = ok & (ratio > 3.3)
    kink = ok & (np.abs(T - 1000.0) < 0.005)
    plain = ok & (np.arange(n) >= 4352)
    print("one-step acceptance: band cells %d (min evaluations %d), range-switch cells %d (min %d), "
          "ordinary cells accepted %.3f" % (band.sum(), itg[band].min(), kink.sum(), itg[kink].min(),
                                            float((itg[plain] == 1).mean())))
    assert band.sum() > 200 and np.all(itg[band] >= 2)
    assert kink.sum() > 200 and np.all(itg[kink] >= 2)
    assert (itg[plain] == 1).mean() > 0.8


@pytest.mark.parametrize("n,band_frac", [(1, 1.0), (31, 0.5), (255, 1.0), (256, 1.0), (257, 0.3), (1000, 1.0),
                                         (4099, 0.2)])
def test_T_from_h_fp64_ragged_sizes(ctx, orc, species, cuda, n, band_frac):
    """The FP64 inversion on ragged sizes, with a share of pseudo-boiling
    cells (O2 at 10 MPa between 150 and 175 K, which take the full
    iteration after the first FP64 evaluation) mixed among ordinary cells,
    up to all of them: every cell's T equals the oracle's inversion and the
    true T to 1e-10, whether it finished after one evaluation, in a full batch
    of its block or in the block's last, partial batch."""
    import torch
    rng = np.random.default_rng(500 + n)
    T, p, Y = W.uniform_cells(n, seed=600 + n)
    band = rng.random(n) < band_frac
    k_o2 = W.SPECIES.index("O2")
    Y[:, band] = 0.0
    Y[k_o2, band] = 1.0
    T[band] = rng.uniform(150.0, 175.0, int(band.sum()))
    p[band] = 10e6
    hs, sts = orc.props(species, T, p, Y)
    guess = T * (1 + rng.uniform(-0.05, 0.05, n))
    To, sto, _ = orc.T_from_h(species, hs[2], p, Y, guess)
    d64 = lambda a: to_dev(a, torch.float64, cuda)
    Tg, stg, itg = ctx.T_from_h(d64(hs[2]), d64(p), d64(Y), d64(guess))
    Tg, stg, itg = Tg.cpu().numpy(), stg.cpu().numpy(), itg.cpu().numpy()
    ok = (sto == 0) & (sts == 0) & (np.abs(T - 1000.0) > 1e-4)   # off the NASA-7 range switch's two roots
    assert ok.sum() >= 0.95 * n
    assert np.all(stg[ok] == 0)
    np.testing.assert_allclose(Tg[ok], To[ok], rtol=1e-10)
    np.testing.assert_allclose(Tg[ok], T[ok], rtol=1e-10)
    # cells well inside the band (cp > 3.3 x the ideal-gas cp) never stop
    # after one evaluation
    dT = 1e-3 * T
    ratio = hs[3] / ((orc.h_ideal(species, T + dT, Y) - orc.h_ideal(species, T - dT, Y)) / (2 * dT))
    inside = ok & band & (ratio > 3.3)
    assert np.all(itg[inside] >= 2)


def test_mixed_inversion_fp64_in_pseudo_boiling_band(ctx, orc, species, cuda):
    """The mixed inversion re-solves in FP64 the cells whose cp exceeds three
    times the ideal-gas cp (the pseudo-boiling band near the pseudo-critical
    line): there its T equals the FP64 inversion's to FP32 rounding, on
    O2 and CH4 across their pseudo-boiling temperatures at 10 MPa and on
    near-pure LOX and CH4 mixtures.  Outside the band it stays the FP32
    iteration, within the FP32 error budget."""
    import torch
    rng = np.random.default_rng(31)
    n = 4096
    k_o2, k_ch4 = W.SPECIES.index("O2"), W.SPECIES.index("CH4")
    Y = np.zeros((9, n))
    T = np.empty(n)
    half = n // 2
    Y[k_o2, :half] = 1.0
    T[:half] = rng.uniform(140.0, 200.0, half)               # O2: Tc 154.6 K
    Y[k_ch4, half:] = 1.0
    T[half:] = rng.uniform(190.0, 280.0, n - half)           # CH4: Tc 190.6 K
    mix = rng.uniform(0, 1, n) < 0.3                         # a trace of products on some cells
    Y[:, mix] = 0.97 * Y[:, mix] + 0.03 * W.dirichlet_half(rng, 9, int(mix.sum()))
    p = np.full(n, 10e6)
    Tt = np.clip(T * (1 + rng.uniform(-0.03, 0.03, n)), 100.0, 3500.0)
    d64 = lambda a: to_dev(a, torch.float64, cuda)
    hs, st0 = ctx.props(d64(Tt), d64(p), d64(Y), outputs=("h", "cp"))
    assert int((st0 != 0).sum()) == 0
    # the FP64 reference sees the same FP32-rounded inputs as the mixed path
    f32 = lambda a: to_dev(a, torch.float32, cuda)
    h32, p32, Y32, T32 = hs[2].float().contiguous(), f32(p), f32(Y), f32(T)
    T64, s64, _ = ctx.T_from_h(h32.double(), p32.double(), Y32.double(), T32.double(), "fp64")
    Tm, sm, _ = ctx.T_from_h(h32, p32, Y32, T32, "mixed", rtol=1e-10)
    Tf, sf, _ = ctx.T_from_h(h32, p32, Y32, T32, "fp32", rtol=1e-10)
    T64, s64, Tm, sm, Tf = (a.cpu().numpy() for a in (T64, s64, Tm, sm, Tf))
    # the band, from the FP64 path's cp and the oracle's ideal-gas enthalpy
    cp = hs[3].cpu().numpy()
    dT = 1e-3 * Tt
    cp_ig = (orc.h_ideal(species, Tt + dT, Y) - orc.h_ideal(species, Tt - dT, Y)) / (2 * dT)
    ratio = cp / cp_ig
    ok = (s64 == 0) & (sm == 0)
    assert ok.mean() > 0.99
    band = ok & (ratio > 3.3)
    out = ok & (ratio < 2.7)
    assert band.sum() > 300 and out.sum() > 300
    e_m = np.abs(Tm.astype(np.float64) - T64) / T64
    e_f = np.abs(Tf.astype(np.float64) - T64) / T64
    print("band cells", int(band.sum()), "mixed max", e_m[band].max(), "fp32 max", e_f[band].max())
    assert e_m[band].max() < 1.2e-7                           # FP64 result rounded to FP32
    assert np.median(e_m[out]) < 1e-5 and e_m[out].max() < 1e-3


# ------------------------------------------- psi and thermal diffusivity
def _psi_condition(orc, species, T, p, Y, idx, h=1e-7):
    """Componentwise condition number of the oracle's psi in (T, p, Y_k)."""
    base, _ = orc.props_ext(species, T[idx], p[idx], Y[:, idx])
    kap = np.zeros(idx.size)
    for which in ["T", "p"] + list(range(Y.shape[0])):
        qs = []
        for sgn in (1.0, -1.0):
            Tt, pt, Yt = T[idx].copy(), p[idx].copy(), Y[:, idx].copy()
            if which == "T":
                Tt *= 1 + sgn * h
            elif which == "p":
                pt *= 1 + sgn * h
            else:
                Yt[which] *= 1 + sgn * h
            q, _ = orc.props_ext(species, Tt, pt, Yt)
            qs.append(q[6])
        kap += np.nan_to_num(np.abs(qs[0] - qs[1]) / (2 * h * np.abs(base[6])), nan=0.0, posinf=0.0)
    return kap


def test_props_ext_psi_alpha_fp64(ctx, orc, species, cuda):
    """pr_props_ext in FP64 against the oracle on uniform cells and the 32^3
    flame-vortex field: psi within 1e-10 (or within its input sensitivity,
    1e-10 + 1e3 eps k_psi, where the oracle shows it ill-conditioned), alpha
    within the GPU's own lambda and cp errors plus 1e-12, the first six
    outputs identical to pr_props'; near-critical roots (cond > 1e4) are
    left out as for cp."""
    import torch
    from .parity import EPS
    T1, p1, Y1 = W.uniform_cells(8192, seed=41)
    T2, p2, Y2 = W.flame_vortex_field(32)[:3]
    T, p, Y = np.concatenate([T1, T2]), np.concatenate([p1, p2]), np.concatenate([Y1, Y2], axis=1)
    d = lambda a: to_dev(a, torch.float64, cuda)
    g8, gs = ctx.props_ext(d(T), d(p), d(Y))
    g6, _ = ctx.props(d(T), d(p), d(Y))
    g8, gs, g6 = g8.cpu().numpy(), gs.cpu().numpy(), g6.cpu().numpy()
    assert np.array_equal(g8[:6], g6, equal_nan=True)
    o, ost, cond = oracle_props(orc, species, T, p, Y)
    o8, ost8 = orc.props_ext(species, T, p, Y)
    assert np.array_equal(o8[:6], o, equal_nan=True) and np.array_equal(ost8, ost)
    well = (ost == 0) & (gs == 0) & (cond <= 1e4)
    assert well.sum() > 40000
    rel = lambda q: np.abs(g8[q] - o8[q]) / np.abs(o8[q])
    e_psi, e_alpha = rel(6), rel(7)
    assert np.all(e_alpha[well] <= 1e-12 + rel(5)[well] + rel(3)[well])
    idx = np.nonzero(well & (e_psi > 1e-10))[0]
    print("psi cells above 1e-10:", idx.size, "of", int(well.sum()), "max", e_psi[well].max())
    assert idx.size < 0.01 * well.sum()
    if idx.size:
        kap = _psi_condition(orc, species, T, p, Y, idx)
        assert np.all(e_psi[idx] <= 1e-10 + 1e3 * EPS * kap)
    # status and NaNs as pr_props
    bad = (ost != 0) & (ost != 5)
    assert np.all(np.isnan(g8[6:, bad]))


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_props_ext_reduced_precision(ctx, orc, species, cuda, precision):
    import torch
    T, p, Y = W.flame_vortex_field(32)[:3]
    T32, p32, Y32 = (a.astype(np.float32).astype(np.float64) for a in (T, p, Y))
    d = lambda a: to_dev(a, torch.float32, cuda)
    g, gs = ctx.props_ext(d(T32), d(p32), d(Y32), precision=precision)
    g, gs = g.cpu().numpy().astype(np.float64), gs.cpu().numpy()
    o, ost = orc.props_ext(species, T32, p32, Y32)
    ok = (ost == 0) & (gs == 0)
    for q, name in ((6, "psi"), (7, "alpha")):
        e = np.abs(g[q, ok] - o[q, ok]) / np.abs(o[q, ok])
        print(precision, name, np.median(e), np.percentile(e, 99))
        assert np.median(e) < 1e-5 and np.percentile(e, 99) < 1e-3


def test_measured_pipe_peaks(prlib, cuda):
    """The pipe microbenchmarks: DFMA throughput near the unit-count figure
    (152 SMs x 2 DFMA/clk x 2 flops at 1.5-2.1 GHz), FP32 FMA far above it
    (GB300's FP64 rate is 1/64 of FP32), and a positive exp2 rate."""
    from paper_2312_04830_gb300 import binding
    fp64 = binding.measure_peak("fp64_fma")
    fp32 = binding.measure_peak("fp32_fma")
    ex2 = binding.measure_peak("mufu_ex2")
    print("measured peaks: FP64 %.3f TFLOP/s, FP32 %.1f TFLOP/s, ex2 %.3g /s" % (fp64 / 1e12, fp32 / 1e12, ex2))
    assert 152 * 4 * 1.5e9 * 0.8 < fp64 < 152 * 4 * 2.1e9 * 1.05
    assert fp32 > 30 * fp64
    assert ex2 > 1e12
    with pytest.raises(binding.PrError):
        binding.check(prlib.pr_measure_peak(9, None), "pr_measure_peak")


def test_mixed_selects_roots_in_fp64(ctx, orc, species, cuda):
    """Subcritical O2 and CH4 (3 MPa, across their saturation temperatures),
    where the cubic has liquid and vapour roots and the residual Gibbs energy
    picks one: the mixed path's FP64 selection keeps the FP64 path's phase on
    every cell (Z within 1e-5), including the cells closest to the switch."""
    import torch
    cells = []
    for name, lo, hi in (("O2", 120.0, 150.0), ("CH4", 150.0, 188.0)):
        k = W.SPECIES.index(name)
        T = np.linspace(lo, hi, 4001)
        Y = np.zeros((9, T.size))
        Y[k] = 1.0
        cells.append((T, Y))
    T = np.concatenate([c[0] for c in cells]).astype(np.float32).astype(np.float64)
    Y = np.concatenate([c[1] for c in cells], axis=1)
    p = np.full(T.size, 3e6)
    _, _, d = orc.diagnose(species, T, p, Y)
    three = np.array([di["n_phys"] for di in d]) >= 2
    assert three.sum() > 1000                   # the FP64 selection is exercised
    g64, s64 = run_props(ctx, T, p, Y, cuda, precision="fp64")
    gm, sm = run_props(ctx, T, p, Y, cuda, precision="mixed")
    ok = (s64 == 0) & (sm == 0)
    assert ok.sum() > 0.99 * T.size
    dz = np.abs(gm[1, ok] - g64[1, ok]) / g64[1, ok]
    print("mixed vs FP64 Z on two-root cells: max", dz[three[ok]].max())
    assert dz.max() < 1e-5
