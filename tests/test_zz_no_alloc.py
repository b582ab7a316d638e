"""pr_fallback_props_noalloc: the fallback evaluation for callers that cannot
allocate device memory (e.g. a host code whose device memory all comes from
its own pool, so the library may not call cudaMalloc on its behalf).  It is
checked against the regular entry point that uses allocated scratch --
surrogate_infer, whose cells outside the training hull take the same FP64
Peng-Robinson step -- bit for bit, and against the FP64 oracle; a table of
more than 9 species takes the padded 32-species kernels.

Collected last on purpose (file name): if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2312_04830_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PR_NOALLOC_MAX_CELLS = 1 << 20
# the outputs are FP32 roundings of FP64 values that match the oracle to 1e-10
ORACLE_TOL = 1e-6


def _noalloc_fn(lib):
    f = lib.pr_fallback_props_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, ctypes.c_int64, vp, vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int64, vp]
    f.restype = ctypes.c_int
    return f


def _cells(n, seed):
    """Cells inside and outside a hull fitted to T in [300, 3100] K."""
    T, p, Y = W.uniform_cells(n, seed=seed)
    T = 300.0 + (T - 100.0) * (2800.0 / 3400.0)
    rng = np.random.default_rng(seed + 1)
    hot = rng.uniform(size=n) < 0.15
    cold = rng.uniform(size=n) < 0.10
    T[hot] = 4300.0
    T[cold & ~hot] = 65.0
    return np.vstack([T, p, Y]).astype(np.float32)


def _rel(out, ref, T):
    scale = np.abs(ref).copy()
    scale[2] = np.maximum(scale[2], np.abs(ref[3]) * T)
    return np.abs(out - ref) / scale


def _call(fn, ctx, T, p, Y, mask, out, stream):
    from paper_2312_04830_gb300 import binding
    rc = fn(ctx.handle, T.numel(), T.data_ptr(), p.data_ptr(), Y.data_ptr(), Y.stride(0), mask.data_ptr(),
            out.data_ptr(), out.stride(0), stream)
    assert rc == 0, binding.lib().pr_last_error()


def _check_oracle(orc, sp, xs64, o, sel, what):
    """FP32 outputs of the selected cells against the FP64 oracle; cells the
    oracle cannot evaluate must be NaN."""
    T, p, Y = xs64[0][sel], xs64[1][sel], xs64[2:][:, sel]
    ref, st = orc.props(sp, T, p, Y)
    good = (st == 0) | (st == 5)
    assert good.sum() > 0.5 * sel.sum(), what
    err = _rel(o[:, sel][:, good], ref[:, good], T[good])
    assert np.all(err <= ORACLE_TOL), (what, float(np.nanmax(err)))
    assert np.all(np.isnan(o[:, sel][:, ~good])), what


def test_noalloc_fallback_matches_surrogate_infer(prlib, orc, cuda, species):
    import torch
    from paper_2312_04830_gb300 import binding
    ctx = binding.PropertyContext(species)
    sg = binding.Surrogate(ctx, width=128, hidden_layers=2, max_batch=256, infer_chunk=1024, seed=3)
    # hull: fitted to a pool of in-range states (targets from the FP64 path)
    Tp, pp, Yp = W.uniform_cells(4000, seed=31)
    Tp = 300.0 + (Tp - 100.0) * (2800.0 / 3400.0)
    d64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=cuda)
    props, st = ctx.props(d64(Tp), d64(pp), d64(Yp))
    keep = ((st == 0) & torch.all(torch.isfinite(props), dim=0) & torch.all(props[[0, 3, 4, 5]] > 0, dim=0))
    x = torch.as_tensor(np.vstack([Tp, pp, Yp]), dtype=torch.float32, device=cuda)[:, keep].contiguous()
    y = props.float()[:, keep].contiguous()
    sg.fit_normalization(x, y)
    fn = _noalloc_fn(binding.lib())
    stream = torch.cuda.current_stream().cuda_stream

    # two calls in a row: the second must not see the first call's list
    for call, (n, seed) in enumerate(((3000, 41), (1777, 43))):
        xs = _cells(n, seed)
        xd = torch.as_tensor(xs, device=cuda)
        T, p, Y = xd[0].contiguous(), xd[1].contiguous(), xd[2:].contiguous()
        ref, flags = sg.infer(T, p, Y)                    # regular path, allocated scratch
        out = torch.full((6, n), -7.0, dtype=torch.float32, device=cuda)
        _call(fn, ctx, T, p, Y, flags, out, stream)
        torch.cuda.synchronize()
        sg.sync_status()
        f = flags.cpu().numpy().astype(bool)
        assert f.sum() > 0.15 * n
        o, r = out.cpu().numpy(), ref.cpu().numpy()
        # the same per-cell step as the surrogate's fallback kernel: the same bits
        same = (o[:, f] == r[:, f]) | (np.isnan(o[:, f]) & np.isnan(r[:, f]))
        assert np.all(same), (call, int((~same).sum()))
        assert np.all(o[:, ~f] == -7.0), "cells outside the mask must be left untouched"
        _check_oracle(orc, species, xs.astype(np.float64), o.astype(np.float64), f, f"call {call}")

    # every mask bit set: every cell is evaluated
    n = 2048
    xs = _cells(n, 47)
    xd = torch.as_tensor(xs, device=cuda)
    T, p, Y = xd[0].contiguous(), xd[1].contiguous(), xd[2:].contiguous()
    out = torch.full((6, n), -7.0, dtype=torch.float32, device=cuda)
    _call(fn, ctx, T, p, Y, torch.ones(n, dtype=torch.uint8, device=cuda), out, stream)
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    assert not np.any(o == -7.0)
    _check_oracle(orc, species, xs.astype(np.float64), o, np.ones(n, bool), "all cells")

    # sizes beyond the fixed scratch capacity are refused before any launch
    rc = fn(ctx.handle, PR_NOALLOC_MAX_CELLS + 1, T.data_ptr(), p.data_ptr(), Y.data_ptr(), PR_NOALLOC_MAX_CELLS + 1,
            flags.data_ptr(), out.data_ptr(), PR_NOALLOC_MAX_CELLS + 1, None)
    assert rc == -1
    assert b"scratch capacity" in binding.lib().pr_last_error()
    sg.close()
    ctx.close()


def test_noalloc_fallback_padded_species_table(prlib, orc, cuda):
    """A 17-species table runs the 32-species kernels: masked cells against
    the FP64 oracle and against pr_props in FP64."""
    import torch
    from paper_2312_04830_gb300 import binding
    names = tuple(W.SPECIES) + ("CH4", "CO2", "H2O", "H2", "CO", "O2", "O", "H")
    sp = W.SpeciesTable(names)
    ctx = binding.PropertyContext(sp)
    fn = _noalloc_fn(binding.lib())
    rng = np.random.default_rng(17)
    n = 3001
    T = rng.uniform(100, 3500, n)
    p = 1e7 * rng.uniform(0.95, 1.05, n)
    Y = rng.dirichlet(np.full(len(names), 0.5), n).T
    xs = np.vstack([T, p, Y]).astype(np.float32)
    xd = torch.as_tensor(xs, device=cuda)
    Td, pd, Yd = xd[0].contiguous(), xd[1].contiguous(), xd[2:].contiguous()
    mask = torch.as_tensor(rng.uniform(size=n) < 0.4, dtype=torch.uint8, device=cuda)
    out = torch.full((6, n), -7.0, dtype=torch.float32, device=cuda)
    _call(fn, ctx, Td, pd, Yd, mask, out, torch.cuda.current_stream().cuda_stream)
    ref, st = ctx.props(Td.double(), pd.double(), Yd.double())
    torch.cuda.synchronize()
    f = mask.cpu().numpy().astype(bool)
    o = out.cpu().numpy().astype(np.float64)
    assert np.all(o[:, ~f] == -7.0)
    _check_oracle(orc, sp, xs.astype(np.float64), o, f, "17 species")
    r = ref.cpu().numpy()
    ok = f & (st.cpu().numpy() == 0)
    err = _rel(o[:, ok], r[:, ok], xs[0].astype(np.float64)[ok])
    assert np.all(err <= ORACLE_TOL), float(err.max())
    ctx.close()
