"""Parity of the per-species outputs (h_k/(R T), mixture-averaged D_k with the
high-pressure correction table) with the FP64 oracle, through the C ABI."""
import ctypes

import numpy as np
import pytest

from paper_2312_04830_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def ctx(prlib, cuda, species):
    from paper_2312_04830_gb300 import binding
    c = binding.PropertyContext(species)
    yield c
    c.close()


def dev(a, dt, cuda):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=cuda)


def run(ctx, T, p, Y, cuda, precision="fp64"):
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    hk, dk, st = ctx.species_props(dev(T, dt, cuda), dev(p, dt, cuda), dev(Y, dt, cuda), precision=precision)
    torch.cuda.synchronize()
    return hk.double().cpu().numpy(), dk.double().cpu().numpy(), st.cpu().numpy()


def assert_parity(g, o, gst, ost, label):
    ghk, gdk = g
    ohk, odk = o
    assert np.array_equal(gst, ost), f"{label}: status differs"
    ok = ost == 0
    assert np.all(np.isnan(ghk[:, ~ok])) and np.all(np.isnan(gdk[:, ~ok]))
    ehk = np.abs(ghk[:, ok] - ohk[:, ok]) / np.maximum(np.abs(ohk[:, ok]), 1.0)
    edk = np.abs(gdk[:, ok] - odk[:, ok]) / np.abs(odk[:, ok])
    assert ehk.max(initial=0) <= RTOL, f"{label}: hk_RT rel err {ehk.max():.3e}"
    assert edk.max(initial=0) <= RTOL, f"{label}: D_k rel err {edk.max():.3e}"
    return float(ehk.max(initial=0)), float(edk.max(initial=0))


def test_species_fp64_uniform_cells(ctx, orc, species, cuda):
    T, p, Y = W.uniform_cells(32768, seed=201)
    g = run(ctx, T, p, Y, cuda)
    hk, dk, st = orc.species_props(species, T, p, Y)
    print(assert_parity(g[:2], (hk, dk), g[2], st, "uniform"))


def test_species_fp64_flame_field_and_pressures(ctx, orc, species, cuda):
    """The flame-vortex field (pure O2 and pure CH4 cells take the
    self-diffusion branch) at 0.1, 1 and 10 MPa."""
    T, p, Y = W.flame_vortex_field(32)
    for scale in (0.01, 0.1, 1.0):
        g = run(ctx, T, p * scale, Y, cuda)
        hk, dk, st = orc.species_props(species, T, p * scale, Y)
        assert_parity(g[:2], (hk, dk), g[2], st, f"field x{scale}")


@pytest.mark.parametrize("n", [1, 127, 129, 40961])
def test_species_fp64_ragged_and_strided(ctx, orc, species, cuda, n):
    import torch
    T, p, Y = W.uniform_cells(n, seed=202 + n)
    Yw = torch.zeros((9, n + 37), dtype=torch.float64, device=cuda)
    Yw[:, :n] = dev(Y, torch.float64, cuda)
    hk, dk, st = ctx.species_props(dev(T, torch.float64, cuda), dev(p, torch.float64, cuda), Yw[:, :n])
    torch.cuda.synchronize()
    o = orc.species_props(species, T, p, Y)
    assert_parity((hk.cpu().numpy(), dk.cpu().numpy()), o[:2], st.cpu().numpy(), o[2], f"n={n}")


def test_species_empty_subsets_and_bad_input(ctx, orc, species, cuda):
    import torch
    from paper_2312_04830_gb300 import binding
    e = torch.empty(0, dtype=torch.float64, device=cuda)
    ctx.species_props(e, e, torch.empty((9, 0), dtype=torch.float64, device=cuda))
    T = np.array([300.0, -1.0, 300.0, np.nan, 800.0])
    p = np.full(5, 1e6)
    Y = np.full((9, 5), 1.0 / 9)
    Y[0, 2] = 0.5
    hk, dk, st = ctx.species_props(dev(T, torch.float64, cuda), dev(p, torch.float64, cuda),
                                   dev(Y, torch.float64, cuda), hk=False)
    assert hk is None
    o = orc.species_props(species, T, p, Y)
    assert list(st.cpu().numpy()) == [0, 4, 4, 4, 0]
    d = dk.cpu().numpy()
    assert np.all(np.isnan(d[:, 1:4]))
    assert np.allclose(d[:, [0, 4]], o[1][:, [0, 4]], rtol=RTOL, atol=0)
    L = binding.lib()
    Td = dev(T, torch.float64, cuda)
    out = torch.empty((9, 5), dtype=torch.float64, device=cuda)
    r = L.pr_species_props(ctx.handle, 0, 5, Td.data_ptr(), Td.data_ptr(), out.data_ptr(), 5, out.data_ptr(), None,
                           4, None, None)
    assert r == -1   # ldo < n


def test_species_fp64_correction_table(ctx, orc, species, cuda):
    """A bilinear correction table on an uneven grid, cells inside and
    outside it (edge clamping), at pressures from 0.2 to 15 MPa."""
    Tr = np.array([0.5, 0.8, 1.0, 1.1, 1.5, 2.5, 6.0])
    pr = np.array([0.1, 0.6, 1.2, 2.0, 3.5])
    rng = np.random.default_rng(9)
    f = rng.uniform(0.2, 1.0, (Tr.size, pr.size))
    T, p, Y = W.uniform_cells(20000, seed=203)
    p = p * np.exp(rng.uniform(-3.9, 0.4, p.size))
    ctx.set_diffusion_correction(Tr, pr, f)
    try:
        g = run(ctx, T, p, Y, cuda)
    finally:
        ctx.set_diffusion_correction()
    o = orc.species_props(species, T, p, Y, corr=(Tr, pr, f))
    assert_parity(g[:2], o[:2], g[2], o[2], "corr")
    g0 = run(ctx, T, p, Y, cuda)   # removed again
    o0 = orc.species_props(species, T, p, Y)
    assert_parity(g0[:2], o0[:2], g0[2], o0[2], "no corr")


def test_species_correction_table_rejected(ctx):
    from paper_2312_04830_gb300 import binding
    good = (np.array([0.5, 1.0]), np.array([0.1, 1.0]), np.ones((2, 2)))
    bad = [(np.array([0.5]), np.array([0.1, 1.0]), np.ones((1, 2))),
           (np.array([1.0, 0.5]), good[1], good[2]),
           (good[0], np.array([0.1, 0.1]), good[2]),
           (good[0], good[1], np.array([[1.0, -0.1], [1.0, 1.0]])),
           (good[0], good[1], np.array([[1.0, np.nan], [1.0, 1.0]]))]
    for t in bad:
        with pytest.raises(binding.PrError):
            ctx.set_diffusion_correction(*t)
    ctx.set_diffusion_correction(*good)
    ctx.set_diffusion_correction()


@pytest.mark.parametrize("names", [("O2",), ("CH4", "O2"),
                                   tuple(W.SPECIES) + ("CH4", "CO2", "H2O", "H2", "CO", "O2", "O", "H")])
def test_species_fp64_species_counts(prlib, orc, cuda, names):
    """1, 2 and 17 species (padded 9- and 32-species kernels)."""
    from paper_2312_04830_gb300 import binding
    sp = W.SpeciesTable(names)
    c = binding.PropertyContext(sp)
    rng = np.random.default_rng(len(names) + 50)
    n = 3000
    T = rng.uniform(100, 3500, n)
    p = 1e7 * rng.uniform(0.95, 1.05, n)
    Y = rng.dirichlet(np.full(len(names), 0.5), n).T.copy()
    g = run(c, T, p, Y, cuda)
    o = orc.species_props(sp, T, p, Y)
    assert_parity(g[:2], o[:2], g[2], o[2], f"N={len(names)}")
    c.close()


def test_species_fp32_error_budget(ctx, orc, species, cuda):
    """FP32 (and PR_MIXED, the same arithmetic here) against the FP64 oracle
    on the FP32-rounded inputs."""
    T, p, Y = W.uniform_cells(32768, seed=204)
    r = lambda a: a.astype(np.float32).astype(np.float64)
    T, p, Y = r(T), r(p), r(Y)
    o = orc.species_props(species, T, p, Y)
    for prec in ("fp32", "mixed"):
        hk, dk, st = run(ctx, T, p, Y, cuda, precision=prec)
        m = (st == 0) & (o[2] == 0)
        assert m.sum() > 32000
        ehk = np.abs(hk[:, m] - o[0][:, m]) / np.maximum(np.abs(o[0][:, m]), 1.0)
        edk = np.abs(dk[:, m] - o[1][:, m]) / o[1][:, m]
        print(prec, "hk median/p99/max", np.median(ehk), np.percentile(ehk, 99), ehk.max(),
              "Dk", np.median(edk), np.percentile(edk, 99), edk.max())
        assert np.median(ehk) < 1e-6 and np.percentile(ehk, 99) < 1e-5
        assert np.median(edk) < 1e-6 and np.percentile(edk, 99) < 1e-5


def test_species_fp32_near_pure_cells(ctx, orc, species, cuda):
    """FP32 on the flame field, whose cells run from pure O2 to pure CH4 through
    mass fractions within an FP32 ulp of 1: no cancellation in 1 - Y_k."""
    T, p, Y = W.flame_vortex_field(32)
    r = lambda a: a.astype(np.float32).astype(np.float64)
    T, p, Y = r(T), r(p), r(Y)
    o = orc.species_props(species, T, p, Y)
    hk, dk, st = run(ctx, T, p, Y, cuda, precision="fp32")
    m = (st == 0) & (o[2] == 0)
    assert m.all()
    edk = np.abs(dk[:, m] - o[1][:, m]) / o[1][:, m]
    print("flame field FP32 D_k max rel err", edk.max())
    assert edk.max() < 1e-5


def test_species_full_field_sampled(ctx, orc, species, cuda):
    """The 128^3 flame-vortex field in one launch; 20000 sampled cells against
    the oracle."""
    import torch
    T, p, Y = W.flame_vortex_field(128)
    hk, dk, st = ctx.species_props(dev(T, torch.float64, cuda), dev(p, torch.float64, cuda),
                                   dev(Y, torch.float64, cuda))
    torch.cuda.synchronize()
    idx = np.random.default_rng(11).choice(T.size, 20000, replace=False)
    idx_t = torch.as_tensor(idx, device=cuda)
    g = (hk[:, idx_t].cpu().numpy(), dk[:, idx_t].cpu().numpy())
    o = orc.species_props(species, T[idx], p[idx], Y[:, idx])
    assert_parity(g, o[:2], st[idx_t].cpu().numpy(), o[2], "128^3 sample")


def test_bilger_z_matches_oracle(ctx, orc, species, cuda):
    """pr_bilger_z against the oracle's element-mass-fraction form: the
    flame-vortex field and random compositions, FP64 and FP32."""
    import torch
    ctx.set_bilger(W.ATOMS_CHO, W.Y_FUEL, W.Y_OX)
    _, _, Yf = W.flame_vortex_field(24)
    Yr = W.dirichlet_half(np.random.default_rng(3), 9, 5000)
    for Y in (Yf, Yr):
        ref = orc.bilger_z(species, W.ATOMS_CHO, W.Y_FUEL, W.Y_OX, Y)
        z64 = ctx.bilger_z(dev(Y, torch.float64, cuda)).cpu().numpy()
        assert np.allclose(z64, ref, rtol=0, atol=1e-14)
        z32 = ctx.bilger_z(dev(Y, torch.float32, cuda), precision="fp32").cpu().numpy().astype(np.float64)
        assert np.allclose(z32, ref, rtol=0, atol=2e-6)
