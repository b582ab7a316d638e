"""Continuous-batching server (GPU): results identical alone and in a mix of
concurrent requests, equal to the direct library calls, admission within the
HBM budget, and bounded waits."""
import numpy as np
import pytest

from paper_2312_04830_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(prlib, cuda, species):
    import torch
    from paper_2312_04830_gb300 import binding
    ctx = binding.PropertyContext(species)
    sg = binding.Surrogate(ctx, width=128, hidden_layers=2, max_batch=256, infer_chunk=8192, seed=5)
    T, p, Y = W.training_states(20000, seed=3)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=cuda)
    props, st = ctx.props(d(T), d(p), d(Y))
    keep = (st == 0) & torch.all(torch.isfinite(props), dim=0) & torch.all(props[[0, 3, 4, 5]] > 0, dim=0)
    x = torch.as_tensor(np.vstack([T, p, Y]), dtype=torch.float32, device=cuda)[:, keep].contiguous()
    sg.fit_normalization(x, props.float()[:, keep].contiguous())
    yield ctx, sg
    sg.close()
    ctx.close()


def make_request(ctx, n, seed, cuda):
    """FP32 host arrays of n cells: T, p, Y and h* = h(T (1 +- 5 %)) from the FP64 path."""
    import torch
    T, p, Y = W.uniform_cells(n, seed=seed)
    T = 300.0 + (T - 100.0) * (2800.0 / 3400.0)
    Tt = W.newton_targets(T, seed=seed + 1)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=cuda)
    hs, _ = ctx.props(d(Tt), d(p), d(Y), outputs=("h",))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return {"T": f32(T), "p": f32(p), "Y": f32(Y), "h": f32(hs[2].cpu().numpy())}


def direct(ctx, sg, req, kind, cuda):
    import torch
    d = lambda a: torch.as_tensor(a, device=cuda)
    if kind == 0:
        out, _ = sg.infer(d(req["T"]), d(req["p"]), d(req["Y"]))
        return out.cpu().numpy()
    Tn, st, _ = ctx.T_from_h(d(req["h"]), d(req["p"]), d(req["Y"]), d(req["T"]), precision="mixed", rtol=1e-6)
    return Tn.cpu().numpy()


def submit(srv, req, kind):
    n = req["T"].size
    if kind == 0:
        out = np.zeros((6, n), dtype=np.float32)
        return srv.submit_props(req["T"], req["p"], req["Y"], out), out
    out = np.zeros(n, dtype=np.float32)
    status = np.zeros(n, dtype=np.int32)
    return srv.submit_T_from_h(req["h"], req["p"], req["Y"], req["T"], out, status), out


def test_same_alone_and_in_mix(setup, cuda):
    from paper_2312_04830_gb300 import serving
    ctx, sg = setup
    srv = serving.Server(ctx, sg, chunk=4096, max_slots=8, budget_bytes=512 << 20)
    R = make_request(ctx, 20000, 101, cuda)
    t, alone = submit(srv, R, 0)
    st, res, lat = srv.wait(t)
    assert st == 0 and res == 0
    reqs = [(make_request(ctx, n, 200 + i, cuda), i % 3 == 2) for i, n in
            enumerate([777, 30000, 5000, 12345, 4096, 60000, 1, 9999, 20000, 333, 15000])]
    tickets = []
    for i, (rq, newton) in enumerate(reqs):
        tickets.append((submit(srv, rq, 1 if newton else 0), rq, newton))
        if i == 5:
            tickets.append((submit(srv, R, 0), R, False))     # R again, in the middle of the mix
    for (t, out), rq, newton in tickets:
        st, res, lat = srv.wait(t)
        assert st == 0 and res == 0
    # direct calls only once the server is idle: the model's buffers are shared
    for (t, out), rq, newton in tickets:
        assert np.array_equal(out, direct(ctx, sg, rq, 1 if newton else 0, cuda), equal_nan=True)
    mixed_R = [out for (t, out), rq, nw in tickets if rq is R][0]
    assert np.array_equal(mixed_R, alone, equal_nan=True)
    s = srv.stats()
    assert s["completed"] == len(tickets) + 1 and s["batches"] >= 2
    srv.close()


def test_admission_respects_budget(setup, cuda):
    from paper_2312_04830_gb300 import serving
    ctx, sg = setup
    budget = 8 << 20
    srv = serving.Server(ctx, sg, chunk=4096, max_slots=4, budget_bytes=budget)
    reqs = [make_request(ctx, 20000, 300 + i, cuda) for i in range(12)]
    ts = [submit(srv, rq, i % 2) for i, rq in enumerate(reqs)]
    big = make_request(ctx, 200000, 400, cuda)            # needs ~13 MB > 8 MiB
    tb, _ = submit(srv, big, 0)
    for t, _ in ts:
        st, res, _ = srv.wait(t)
        assert st == 0 and res == 0
    st, res, _ = srv.wait(tb)
    assert st == 0 and res == -2                          # PR_ENOMEM: can never fit
    s = srv.stats()
    assert 0 < s["peak_bytes_in_use"] <= budget
    assert s["bytes_in_use"] == 0
    srv.close()


def test_wait_times_out_then_completes(setup, cuda):
    from paper_2312_04830_gb300 import serving
    ctx, sg = setup
    srv = serving.Server(ctx, sg, chunk=8192, max_slots=4, budget_bytes=256 << 20)
    rq = make_request(ctx, 400000, 500, cuda)
    t, out = submit(srv, rq, 1)
    st, _, _ = srv.wait(t, timeout_ms=0.001)
    assert st == -4                                       # PR_ETIMEOUT, request still running
    st, res, lat = srv.wait(t, timeout_ms=120000.0)
    assert st == 0 and res == 0 and lat > 0
    srv.close()


def test_request_precisions_match_direct_calls_and_oracle(setup, orc, species, cuda):
    """Every request precision, both kinds, in one mix: served results equal the
    direct library call of that precision bit for bit (the FP64 paths on the
    widened FP32 inputs, rounded to FP32), and a sample of them -- the FP64
    paths, and the surrogate's FP64 fallback cells outside the hull -- is
    checked against the FP64 oracle."""
    import torch
    from paper_2312_04830_gb300 import serving
    from .parity import rel_errors
    ctx, sg = setup
    srv = serving.Server(ctx, sg, chunk=4096, max_slots=8, budget_bytes=512 << 20)
    reqs = {}
    for j, prec in enumerate(("server", "fp64", "mixed", "fp32")):
        for kind in (0, 1):
            rq = make_request(ctx, 7000 + 911 * j + 37 * kind, 600 + 10 * j + kind, cuda)
            if kind == 0 and prec == "server":
                rq["T"][::5] = 4300.0                   # outside the hull: the FP64 fallback
            n = rq["T"].size
            if kind == 0:
                out = np.zeros((6, n), dtype=np.float32)
                t = srv.submit_props(rq["T"], rq["p"], rq["Y"], out, precision=prec)
            else:
                out = np.zeros(n, dtype=np.float32)
                st = np.zeros(n, dtype=np.int32)
                t = srv.submit_T_from_h(rq["h"], rq["p"], rq["Y"], rq["T"], out, st, precision=prec)
            reqs[(prec, kind)] = (t, rq, out)
    for t, _, _ in reqs.values():
        st_, res, _ = srv.wait(t)
        assert st_ == 0 and res == 0
    srv.close()
    d32 = lambda a: torch.as_tensor(a, device=cuda)
    d64 = lambda a: torch.as_tensor(a.astype(np.float64), device=cuda)
    for (prec, kind), (t, rq, out) in reqs.items():
        if kind == 0:
            if prec == "server":
                exp, fb = sg.infer(d32(rq["T"]), d32(rq["p"]), d32(rq["Y"]))
                fb = fb.cpu().numpy().astype(bool)
                assert fb[::5].all()
            elif prec == "fp64":
                exp, _ = ctx.props(d64(rq["T"]), d64(rq["p"]), d64(rq["Y"]), precision="fp64")
            else:
                exp, _ = ctx.props(d32(rq["T"]), d32(rq["p"]), d32(rq["Y"]), precision=prec)
            exp = exp.float().cpu().numpy()
        else:
            if prec == "fp64":
                Tn, _, _ = ctx.T_from_h(d64(rq["h"]), d64(rq["p"]), d64(rq["Y"]), d64(rq["T"]), precision="fp64",
                                        rtol=1e-12)
            else:
                Tn, _, _ = ctx.T_from_h(d32(rq["h"]), d32(rq["p"]), d32(rq["Y"]), d32(rq["T"]),
                                        precision="mixed" if prec in ("server", "mixed") else "fp32", rtol=1e-6)
            exp = Tn.float().cpu().numpy()
        assert np.array_equal(out, exp, equal_nan=True), (prec, kind)
    # against the oracle (inputs: the FP32 request values, widened)
    x = lambda rq, k: rq[k].astype(np.float64)
    for prec, sel in (("fp64", slice(None, None, 7)), ("server", slice(None, None, 5))):
        t, rq, out = reqs[(prec, 0)]
        o, ost = orc.props(species, x(rq, "T")[sel], x(rq, "p")[sel], x(rq, "Y")[:, sel])
        ok = ost == 0
        assert ok.sum() > 100
        err = rel_errors(out[:, sel].astype(np.float64)[:, ok], o[:, ok], x(rq, "T")[sel][ok])
        assert err.max() < 1e-6, (prec, err.max())
    t, rq, out = reqs[("fp64", 1)]
    sel = slice(None, None, 7)
    Tor, ost, _ = orc.T_from_h(species, x(rq, "h")[sel], x(rq, "p")[sel], x(rq, "Y")[:, sel], x(rq, "T")[sel])
    ok = ost == 0
    assert ok.sum() > 100
    assert np.max(np.abs(out[sel][ok] - Tor[ok]) / Tor[ok]) < 1e-6
