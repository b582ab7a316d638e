"""Python side of the continuous-batching property server (argument marshalling
to serve_create / serve_submit / serve_poll / serve_wait / serve_stats) and a
trace driver for the serving workload: clients with flame-vortex fields of
uneven grid sizes submitting forward-property and T-from-h requests with
Poisson arrivals."""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import binding

SV_PROPS, SV_T_FROM_H = 0, 1
SV_PREC = {"server": 0, "fp64": 1, "mixed": 2, "fp32": 3}


class _SvRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("precision", ctypes.c_int32), ("n", ctypes.c_int64),
                ("T", ctypes.c_void_p), ("p", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("h", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class _SvConfig(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int32), ("max_slots", ctypes.c_int32), ("newton_precision", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_size_t)]


class _SvStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "completed", "batches", "slots_used", "slots_launched")] + \
               [("cells", ctypes.c_int64)] + [(f, ctypes.c_size_t) for f in ("bytes_in_use", "peak_bytes_in_use",
                                                                              "queued", "active")]


def _lib():
    L = binding.lib()
    if not getattr(L, "_sv_ready", False):
        vp, i32, u64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
        L.serve_create.argtypes = [vp, vp, ctypes.POINTER(_SvConfig), ctypes.POINTER(vp)]
        L.serve_create.restype = i32
        L.serve_submit.argtypes = [vp, ctypes.POINTER(_SvRequest), ctypes.POINTER(u64)]
        L.serve_submit.restype = i32
        L.serve_poll.argtypes = [vp, u64, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(d)]
        L.serve_poll.restype = i32
        L.serve_wait.argtypes = [vp, u64, d, ctypes.POINTER(i32), ctypes.POINTER(d)]
        L.serve_wait.restype = i32
        L.serve_stats.argtypes = [vp, ctypes.POINTER(_SvStats)]
        L.serve_stats.restype = i32
        L.serve_destroy.argtypes = [vp]
        L.serve_destroy.restype = None
        L._sv_ready = True
    return L


def _addr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous and a.dtype in (np.float32, np.int32)
        return a.ctypes.data
    return a.data_ptr()          # torch CPU tensor (pinned or not)


class Server:
    """serve_create wrapper.  Host arrays of a request must stay alive until it is done."""

    def __init__(self, ctx, model=None, chunk=1 << 18, max_slots=16, budget_bytes=80 << 30,
                 newton_precision="mixed"):
        L = _lib()
        cfg = _SvConfig(chunk, max_slots, binding.PRECISIONS[newton_precision], 0, budget_bytes)
        h = ctypes.c_void_p()
        binding.check(L.serve_create(ctx.handle, model.handle if model is not None else None, ctypes.byref(cfg),
                                     ctypes.byref(h)), "serve_create")
        self.handle = h
        self._keep = {}

    def close(self):
        if getattr(self, "handle", None):
            _lib().serve_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit_props(self, T, p, Y, out, precision="server") -> int:
        n = T.shape[0]
        r = _SvRequest(SV_PROPS, SV_PREC[precision], n, _addr(T), _addr(p), _addr(Y), None, _addr(out), None)
        return self._submit(r, (T, p, Y, out))

    def submit_T_from_h(self, h, p, Y, T_guess, out, status=None, precision="server") -> int:
        n = h.shape[0]
        r = _SvRequest(SV_T_FROM_H, SV_PREC[precision], n, _addr(T_guess), _addr(p), _addr(Y), _addr(h), _addr(out),
                       _addr(status))
        return self._submit(r, (h, p, Y, T_guess, out, status))

    def _submit(self, r, keep):
        t = ctypes.c_uint64()
        binding.check(_lib().serve_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "serve_submit")
        self._keep[t.value] = keep
        return t.value

    def poll(self, ticket):
        done, res, lat = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        binding.check(_lib().serve_poll(self.handle, ticket, ctypes.byref(done), ctypes.byref(res), ctypes.byref(lat)),
                      "serve_poll")
        if done.value:
            self._keep.pop(ticket, None)
            return True, res.value, lat.value
        return False, None, None

    def wait(self, ticket, timeout_ms=60000.0):
        """(status, result, latency_ms); status is PR_ETIMEOUT (-4) if it ran out."""
        res, lat = ctypes.c_int(), ctypes.c_double()
        st = _lib().serve_wait(self.handle, ticket, float(timeout_ms), ctypes.byref(res), ctypes.byref(lat))
        if st == 0:
            self._keep.pop(ticket, None)
        return st, res.value, lat.value

    def stats(self) -> dict:
        s = _SvStats()
        binding.check(_lib().serve_stats(self.handle, ctypes.byref(s)), "serve_stats")
        return {f: getattr(s, f) for f, _ in _SvStats._fields_}


# ------------------------------------------------------------------- driver
def client_field(big, g):
    """A g^3 client field: the nearest cells of a larger flame-vortex field
    (same structure at grid g).  big = dict of host tensors T, p, Y, h."""
    import torch
    G = round(big["T"].numel() ** (1.0 / 3.0))
    ix = torch.as_tensor(np.minimum(((np.arange(g) + 0.5) * G / g).astype(np.int64), G - 1))
    idx = ((ix[:, None, None] * G + ix[None, :, None]) * G + ix[None, None, :]).reshape(-1)
    f = {"T": big["T"][idx], "p": big["p"][idx], "h": big["h"][idx],
         "Y": big["Y"][:, idx].contiguous()}
    return {k: v.pin_memory() for k, v in f.items()}


def run_trace(server, fields, grids, kinds, clients, arrivals, out_pool):
    """Submit the trace at its arrival times (seconds from start); return
    per-request latencies [ms], kinds, cells and the makespan [s]."""
    order = np.argsort(arrivals)
    t0 = time.perf_counter()
    tickets = {}
    for i in order:
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        c = clients[i]
        f = fields[c]
        out = out_pool[c]
        if kinds[i] == SV_PROPS:
            tickets[i] = server.submit_props(f["T"], f["p"], f["Y"], out["props"])
        else:
            tickets[i] = server.submit_T_from_h(f["h"], f["p"], f["Y"], f["T"], out["T"], out["status"])
    lat = np.zeros(len(arrivals))
    for i, t in tickets.items():
        st, res, l = server.wait(t, 600000.0)
        assert st == 0 and res == 0, (st, res)
        lat[i] = l
    makespan = time.perf_counter() - t0
    return lat, makespan
