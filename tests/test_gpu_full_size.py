"""Parity at the full benchmark size (GPU): the 256^3 flame-vortex field
(16,777,216 cells, N = 9) in the launch configuration the benchmark times.

The property evaluation and the inversion run over the whole field in one
call each; sampled cells are checked against the oracle, which the oracle can
compute one by one.  The surrogate runs the whole field in 4 Mi-row chunks;
the fused kernel's outputs equal the per-layer launches bit for bit on every
row, and sampled rows match the float64 forward of the oracle MLP.  Inputs
come from the seeded generators; expected values from the oracle only.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2312_04830_gb300 import workloads as W

from .parity import assert_fp64_parity, root_sensitivity_bound
from .test_gpu_surrogate import h_ig_of, make_pool, standardise, unflatten

pytestmark = pytest.mark.gpu

GRID = 256
N_SAMPLE = 20000
CHUNK = 1 << 22   # rows per fused-inference launch, as in the benchmark


@pytest.fixture(scope="module")
def ctx(prlib, cuda, species):
    from paper_2312_04830_gb300 import binding
    c = binding.PropertyContext(species)
    yield c
    c.close()


@pytest.fixture(scope="module")
def field():
    T, p, Y = W.flame_vortex_field(GRID)
    Ttrue = W.newton_targets(T)
    idx = np.sort(np.random.default_rng(31).choice(T.size, N_SAMPLE, replace=False))
    return T, p, Y, Ttrue, idx


def dev(a, dtype, cuda):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=cuda)


def test_props_fp64_full_field_sampled(ctx, orc, species, cuda, field):
    """pr_props in FP64 over all 16.8 M cells in one call; 20000 sampled cells
    against the oracle (1e-10, with the oracle's sensitivity allowance)."""
    import torch
    T, p, Y, _, idx = field
    out, st = ctx.props(dev(T, torch.float64, cuda), dev(p, torch.float64, cuda), dev(Y, torch.float64, cuda),
                        precision="fp64")
    torch.cuda.synchronize()
    it = torch.as_tensor(idx, device=cuda)
    g, gs = out[:, it].cpu().numpy(), st[it].cpu().numpy()
    assert np.all(st.cpu().numpy() >= 0)
    Ts, ps, Ys = T[idx], p[idx], Y[:, idx]
    o, os_, d = orc.diagnose(species, Ts, ps, Ys)
    tb = orc.Table(species)
    rep = assert_fp64_parity(g, gs, o, os_, Ts, d, label="256^3 sample",
                             zsens=lambda k, Z, dz, oo: root_sensitivity_bound(orc, tb, Ts, ps, Ys, k, Z, dz, oo))
    assert rep["n_ok"] > 0.99 * N_SAMPLE


def test_T_from_h_fp64_full_field_sampled(ctx, orc, species, cuda, field):
    """pr_T_from_h in FP64 over all 16.8 M cells in one call, as the benchmark
    runs it (h* = h(T_true) of the FP64 path, start at the field's T); on
    20000 sampled cells the result equals the oracle's own inversion of its
    own h(T_true) and T_true (1e-10)."""
    import torch
    T, p, Y, Ttrue, idx = field
    T64, p64, Y64 = dev(T, torch.float64, cuda), dev(p, torch.float64, cuda), dev(Y, torch.float64, cuda)
    hs, _ = ctx.props(dev(Ttrue, torch.float64, cuda), p64, Y64, precision="fp64", outputs=("h",))
    hstar = hs[2].clone()
    del hs
    Tg, stg, itg = ctx.T_from_h(hstar, p64, Y64, T64)
    torch.cuda.synchronize()
    it = torch.as_tensor(idx, device=cuda)
    Tg, stg, itg = Tg[it].cpu().numpy(), stg[it].cpu().numpy(), itg[it].cpu().numpy()
    Ts, ps, Ys = T[idx], p[idx], Y[:, idx]
    ho, sth = orc.props(species, Ttrue[idx], ps, Ys)
    To, sto, _ = orc.T_from_h(species, ho[2], ps, Ys, Ts)
    ok = (sto == 0) & (sth == 0)
    assert ok.sum() > 0.99 * N_SAMPLE
    assert np.all(stg[ok] == 0)
    np.testing.assert_allclose(Tg[ok], To[ok], rtol=1e-10)
    np.testing.assert_allclose(Tg[ok], Ttrue[idx][ok], rtol=1e-10)
    assert itg[ok].max() <= 60


def test_surrogate_full_field_fused_equals_layerwise_and_oracle(ctx, orc, species, cuda, field):
    """surrogate_infer over all 16.8 M rows in 4 Mi-row chunks (width 512, 4
    hidden layers): the default kernel (activations resident in shared memory)
    and the L2-ring kernel equal the per-layer launches bit for bit on every
    row, and sampled rows inside the training hull match the float64 forward
    of the same weights."""
    import torch
    from paper_2312_04830_gb300 import binding
    T, p, Y, _, idx = field
    sg = binding.Surrogate(ctx, width=512, hidden_layers=4, max_batch=1024, infer_chunk=CHUNK, seed=41)
    x, y = make_pool(orc, species, 8000, seed=42)
    sg.fit_normalization(dev(x, torch.float32, cuda), dev(y, torch.float32, cuda))
    Td, pd, Yd = dev(T, torch.float32, cuda), dev(p, torch.float32, cuda), dev(Y, torch.float32, cuda)
    assert sg.fused_kind == "resident"
    out_f, fb_f = sg.infer(Td, pd, Yd)
    sg.sync_status()
    sg.set_fused_infer(False)
    out_l, fb_l = sg.infer(Td, pd, Yd)
    sg.sync_status()
    sg.set_fused_infer(True)
    out_r, fb_r = sg.infer(Td, pd, Yd)
    sg.sync_status()
    for o, f in ((out_f, fb_f), (out_r, fb_r)):
        assert torch.equal(f, fb_l)
        assert torch.equal(o.isnan(), out_l.isnan())
        same = (o == out_l) | (o.isnan() & out_l.isnan())
        assert bool(same.all())
    del out_r, fb_r
    it = torch.as_tensor(idx, device=cuda)
    o, fb = out_f[:, it].double().cpu().numpy(), fb_f[it].cpu().numpy()
    keep = fb == 0
    assert keep.mean() > 0.5
    xs = np.vstack([T[idx], p[idx], Y[:, idx]]).astype(np.float32)[:, keep]
    norm = sg.get_normalization().astype(np.float64)
    params = unflatten(sg.get_params(), [13, 512, 512, 512, 512, 6])
    s_in, _ = standardise(xs, np.ones((6, xs.shape[1]), np.float32), norm, species)
    yhat, _ = omlp.forward(params, s_in, "tanh")
    s_gpu = (omlp.output_targets(o[:, keep], h_ig_of(species, xs)) - norm[26:32]) / norm[32:38]
    err = np.abs(s_gpu - yhat)
    print("full field: fallback fraction", 1 - keep.mean(), "standardised error median", np.median(err),
          "max", err.max())
    assert np.median(err) < 0.01
    assert err.max() < 0.1
    sg.close()


def test_props_fp64_64bit_indexing(ctx, orc, species, cuda):
    """Maximum-size edge case: 2^28 + 77 cells in one pr_props call (FP64,
    about 37 GB on the device), so that the species-major mass fractions'
    element index k ldY + i passes 2^31.  The cells tile a seeded set of
    32768; sampled cells near the end and across the range equal the oracle
    on their base cells (1e-10)."""
    import torch
    Tb, pb, Yb = W.uniform_cells(32768, seed=51)
    nb = Tb.size
    n = (1 << 28) + 77
    reps = -(-n // nb)
    Td = dev(Tb, torch.float64, cuda).repeat(reps)[:n].contiguous()
    pd = dev(pb, torch.float64, cuda).repeat(reps)[:n].contiguous()
    Yd = dev(Yb, torch.float64, cuda).repeat(1, reps)[:, :n].contiguous()
    out, st = ctx.props(Td, pd, Yd, precision="fp64")
    torch.cuda.synchronize()
    del Td, pd, Yd
    rng = np.random.default_rng(52)
    idx = np.unique(np.concatenate([np.arange(n - 2000, n), rng.choice(n, 3000, replace=False)]))
    assert 8 * n + idx.max() > (1 << 31)
    it = torch.as_tensor(idx, device=cuda)
    g, gs = out[:, it].cpu().numpy(), st[it].cpu().numpy()
    del out, st
    base = idx % nb
    o, os_, d = orc.diagnose(species, Tb[base], pb[base], Yb[:, base])
    tb = orc.Table(species)
    Tq, pq, Yq = Tb[base], pb[base], Yb[:, base]
    rep = assert_fp64_parity(g, gs, o, os_, Tq, d, label="2^28 + 77 cells",
                             zsens=lambda k, Z, dz, oo: root_sensitivity_bound(orc, tb, Tq, pq, Yq, k, Z, dz, oo))
    assert rep["n_ok"] > 0.97 * idx.size
