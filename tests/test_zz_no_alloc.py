"""pr_fallback_props_noalloc: the fallback evaluation for callers that cannot
allocate device memory (e.g. a host code whose device memory all comes from
its own pool), checked against the regular entry point that uses allocated
scratch -- surrogate_infer, whose cells outside the training hull take the
same FP64 Peng-Robinson step.

Collected last on purpose (file name): if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2312_04830_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PR_NOALLOC_MAX_CELLS = 1 << 20


def _noalloc_fn(lib):
    f = lib.pr_fallback_props_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, ctypes.c_int64, vp, vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int64, vp]
    f.restype = ctypes.c_int
    return f


def _cells(species, n, seed):
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


def test_noalloc_fallback_matches_surrogate_infer(prlib, cuda, species):
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

    for call, (n, seed) in enumerate(((3000, 41), (1777, 43))):
        xs = torch.as_tensor(_cells(species, n, seed), device=cuda)
        T, p, Y = xs[0].contiguous(), xs[1].contiguous(), xs[2:].contiguous()
        ref, flags = sg.infer(T, p, Y)                    # regular path, allocated scratch
        out = torch.full((6, n), -7.0, dtype=torch.float32, device=cuda)
        rc = fn(ctx.handle, n, T.data_ptr(), p.data_ptr(), Y.data_ptr(), Y.stride(0), flags.data_ptr(),
                out.data_ptr(), out.stride(0), torch.cuda.current_stream().cuda_stream)
        assert rc == 0, binding.lib().pr_last_error()
        torch.cuda.synchronize()
        sg.sync_status()
        f = flags.cpu().numpy().astype(bool)
        assert f.sum() > 0.15 * n
        o, r = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        both_nan = np.isnan(o[:, f]) & np.isnan(r[:, f])
        err = np.where(both_nan, 0.0, _rel(o[:, f], r[:, f], xs[0].cpu().numpy().astype(np.float64)[f]))
        assert np.all(err <= 1e-6), (call, np.nanmax(err))
        assert np.all(o[:, ~f] == -7.0), "cells outside the mask must be left untouched"

    # sizes beyond the fixed scratch capacity are refused before any launch
    rc = fn(ctx.handle, PR_NOALLOC_MAX_CELLS + 1, T.data_ptr(), p.data_ptr(), Y.data_ptr(), PR_NOALLOC_MAX_CELLS + 1,
            flags.data_ptr(), out.data_ptr(), PR_NOALLOC_MAX_CELLS + 1, None)
    assert rc == -1
    assert b"scratch capacity" in binding.lib().pr_last_error()
    sg.close()
    ctx.close()
