"""Plain FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library (the CUDA
path) never calls it and shares no code with it.

* ``pr_oracle.c`` -- Peng-Robinson / vdW mixing / NASA-7 / Chung / Newton, and the
  per-species standard-state enthalpies and mixture-averaged diffusion, per
  cell, in FP64 (see the header of that file for the passages it follows).
* ``mlp.py``      -- the surrogate MLP forward, backward and Adam step in
  float64 NumPy.

The C part is compiled with gcc (``-O2 -ffp-contract=off``, OpenMP for the
batch loops, no fast-math) into ``oracle/liborc.so`` on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pr_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

R = 8.314462618

STATUS = {0: "ok", 1: "newton_maxit", 2: "h_out_of_range", 3: "no_root", 4: "bad_input", 5: "ambiguous"}


_OPC_SRC = os.path.join(_HERE, "opcount.cpp")
_OPC_LIB = os.path.join(_HERE, "libopcount.so")
_opc = None


def build_opcount(force: bool = False) -> str:
    """Compile the operation-counting build of the oracle (opcount.cpp, g++)."""
    newest = max(os.path.getmtime(_OPC_SRC), os.path.getmtime(_SRC))
    if force or not os.path.exists(_OPC_LIB) or os.path.getmtime(_OPC_LIB) < newest:
        tmp = _OPC_LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall",
               "-Wno-class-memaccess", "-Wno-unused-function", "-o", tmp, _OPC_SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _OPC_LIB)
    return _OPC_LIB


OP_KINDS = ("add", "mul", "div", "sqrt", "cbrt", "exp", "expm1", "log", "log1p", "pow", "trig", "cmp")
OP_STEPS = {0: "diagnostics", 1: "composition", 2: "species EOS terms", 3: "mixing", 4: "cubic roots",
            5: "root selection", 6: "ideal gas", 7: "departures", 8: "Chung mixture rules",
            9: "Chung dense correlation", 10: "output assembly"}


def op_counts(sp, T, p, Y):
    """Per-cell operation counts of the oracle (mean over the cells that
    evaluate with status 0): {"steps": {name: {kind: count}}, "short":
    {"mixing" | "chung_rules" | "cubic_roots" | "species_terms" | "ideal_gas":
    {kind: count}}, "check": [max relative difference of the five short forms
    from the oracle],
    "cells": n}.  See opcount.cpp for what is counted."""
    global _opc
    with _lock:
        if _opc is None:
            L = ctypes.CDLL(build_opcount())
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            L.orc_count_ops.argtypes = [vp] * 10 + [ctypes.c_int, i64, vp, vp, vp, vp, vp, vp]
            L.orc_count_ops.restype = i64
            _opc = L
    tb = sp if isinstance(sp, Table) else Table(sp)
    a = tb.arrays
    T, p, Y = _soa(T, p, Y, tb.n)
    n = T.size
    nk = len(OP_KINDS)
    counts = np.zeros((16, nk))
    short = np.zeros((5, nk))
    check = np.zeros(5)
    good = _opc.orc_count_ops(*[_ptr(a[k]) for k in ("W", "Tc", "pc", "omega", "Vc", "dipole", "kappa", "nasa_lo",
                                                      "nasa_hi", "T_mid")], tb.n, n, _ptr(T), _ptr(p), _ptr(Y),
                              _ptr(counts), _ptr(short), _ptr(check))
    g = max(int(good), 1)
    steps = {OP_STEPS[s]: dict(zip(OP_KINDS, (counts[s] / g).tolist())) for s in OP_STEPS}
    shorts = {nm: dict(zip(OP_KINDS, (short[r] / g).tolist()))
              for r, nm in enumerate(("mixing", "chung_rules", "cubic_roots", "species_terms", "ideal_gas"))}
    return {"steps": steps, "short": shorts, "check": check.tolist(), "cells": int(good)}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (idempotent)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class Species(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("transport_rule", ctypes.c_int32),
                ("printed_constants", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("W", ctypes.c_void_p), ("Tc", ctypes.c_void_p), ("pc", ctypes.c_void_p),
                ("omega", ctypes.c_void_p), ("Vc", ctypes.c_void_p), ("dipole", ctypes.c_void_p),
                ("kappa", ctypes.c_void_p), ("nasa_lo", ctypes.c_void_p), ("nasa_hi", ctypes.c_void_p),
                ("T_mid", ctypes.c_void_p), ("kij", ctypes.c_void_p)]


class Diag(ctypes.Structure):
    _fields_ = [("Wbar", ctypes.c_double), ("am", ctypes.c_double), ("dam", ctypes.c_double),
                ("d2am", ctypes.c_double), ("bm", ctypes.c_double), ("A", ctypes.c_double),
                ("B", ctypes.c_double), ("roots", ctypes.c_double * 3), ("n_roots", ctypes.c_int32),
                ("n_phys", ctypes.c_int32), ("Z", ctypes.c_double), ("gres_gap", ctypes.c_double),
                ("cond", ctypes.c_double), ("h_ig", ctypes.c_double), ("cp_ig", ctypes.c_double),
                ("cv_ig_molar", ctypes.c_double), ("h_dep", ctypes.c_double), ("cp_dep", ctypes.c_double),
                ("dpdT", ctypes.c_double), ("dpdV", ctypes.c_double), ("mu_dilute", ctypes.c_double),
                ("lambda_dilute", ctypes.c_double), ("cancel_mu", ctypes.c_double), ("cancel_lam", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            L.orc_props.argtypes = [vp, i64, vp, vp, vp, vp, vp, i32]
            L.orc_props.restype = None
            L.orc_props_ext.argtypes = [vp, i64, vp, vp, vp, vp, vp, i32]
            L.orc_props_ext.restype = None
            L.orc_h_ideal.argtypes = [vp, i64, vp, vp, vp]
            L.orc_h_ideal.restype = None
            L.orc_diagnose.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
            L.orc_diagnose.restype = None
            L.orc_props_at_Z.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
            L.orc_props_at_Z.restype = None
            L.orc_chung_pure.argtypes = [d] * 9 + [vp]
            L.orc_chung_pure.restype = None
            L.orc_T_from_h.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, i32, d, i32]
            L.orc_T_from_h.restype = None
            L.orc_cubic_real_roots.argtypes = [d, d, d, vp]
            L.orc_cubic_real_roots.restype = i32
            L.orc_pr_constants.argtypes = [i32, vp, vp]
            L.orc_pr_constants.restype = None
            L.orc_pr_gres.argtypes = [d, d, d]
            L.orc_pr_gres.restype = d
            L.orc_species_props.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, i32]
            L.orc_species_props.restype = None
            L.orc_neufeld_omega_d.argtypes = [d]
            L.orc_neufeld_omega_d.restype = d
            L.orc_bilger_z.argtypes = [i32, vp, vp, vp, vp, i64, vp, vp]
            L.orc_bilger_z.restype = None
            L.orc_max_threads.argtypes = []
            L.orc_max_threads.restype = i32
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Table:
    """Holds the species arrays alive for the C struct."""

    def __init__(self, sp, transport_rule: int = 0, printed_constants: bool = False, use_kij: bool = True):
        self.arrays = dict(
            W=np.ascontiguousarray(sp.W, dtype=np.float64), Tc=np.ascontiguousarray(sp.Tc, dtype=np.float64),
            pc=np.ascontiguousarray(sp.pc, dtype=np.float64), omega=np.ascontiguousarray(sp.omega, dtype=np.float64),
            Vc=np.ascontiguousarray(sp.Vc, dtype=np.float64), dipole=np.ascontiguousarray(sp.dipole, dtype=np.float64),
            kappa=np.ascontiguousarray(sp.kappa, dtype=np.float64),
            nasa_lo=np.ascontiguousarray(sp.nasa_lo, dtype=np.float64),
            nasa_hi=np.ascontiguousarray(sp.nasa_hi, dtype=np.float64),
            T_mid=np.ascontiguousarray(sp.T_mid, dtype=np.float64))
        kij = getattr(sp, "kij", None)
        self.kij = (np.ascontiguousarray(kij, dtype=np.float64) if (use_kij and kij is not None and np.any(kij))
                    else None)
        self.n = int(sp.W.size)
        self.s = Species(self.n, transport_rule, int(printed_constants), 0,
                         *[_ptr(self.arrays[k]) for k in ("W", "Tc", "pc", "omega", "Vc", "dipole", "kappa",
                                                          "nasa_lo", "nasa_hi", "T_mid")],
                         _ptr(self.kij))

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _soa(T, p, Y, n_species):
    T = np.ascontiguousarray(T, dtype=np.float64)
    p = np.ascontiguousarray(np.broadcast_to(p, T.shape), dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(n_species, T.size)
    return T, p, Y


def props(sp, T, p, Y, threads: int = 0, **kw):
    """(out[6, n] = rho, Z, h, cp, mu, lambda; status[n]) for SoA inputs."""
    tb = sp if isinstance(sp, Table) else Table(sp, **kw)
    T, p, Y = _soa(T, p, Y, tb.n)
    n = T.size
    out = np.empty((6, n))
    st = np.empty(n, dtype=np.int32)
    lib().orc_props(tb.ref, n, _ptr(T), _ptr(p), _ptr(Y), _ptr(out), _ptr(st), int(threads))
    return out, st


def props_ext(sp, T, p, Y, threads: int = 0, **kw):
    """(out[8, n] = rho, Z, h, cp, mu, lambda, psi, alpha; status[n])."""
    tb = sp if isinstance(sp, Table) else Table(sp, **kw)
    T, p, Y = _soa(T, p, Y, tb.n)
    n = T.size
    out = np.empty((8, n))
    st = np.empty(n, dtype=np.int32)
    lib().orc_props_ext(tb.ref, n, _ptr(T), _ptr(p), _ptr(Y), _ptr(out), _ptr(st), int(threads))
    return out, st


def h_ideal(sp, T, Y, **kw):
    """Mass-specific ideal-gas enthalpy sum_k Y_k h_k(T) / W_k [J/kg] (NASA-7)."""
    tb = sp if isinstance(sp, Table) else Table(sp, **kw)
    T, _, Y = _soa(T, 0.0, Y, tb.n)
    h = np.empty(T.size)
    lib().orc_h_ideal(tb.ref, T.size, _ptr(T), _ptr(Y), _ptr(h))
    return h


def chung_pure(Tc, Vc, omega, M, dipole, kappa, T, rho_mol, cv_molar):
    """Chung's correlation for one pure fluid at (T, rho_mol): (mu, lambda,
    mu_dilute, lambda_dilute) [Pa s, W/(m K)]; units as the species table."""
    out = np.zeros(4)
    lib().orc_chung_pure(Tc, Vc, omega, M, dipole, kappa, T, rho_mol, cv_molar, _ptr(out))
    return tuple(out)


def props_at_Z(sp, T, p, Y, Z, **kw):
    """(out[6, n], status[n]) with the root Z[i] in place of the selected one:
    the derived outputs as functions of the root (a test aid)."""
    tb = sp if isinstance(sp, Table) else Table(sp, **kw)
    T, p, Y = _soa(T, p, Y, tb.n)
    n = T.size
    Z = np.ascontiguousarray(np.broadcast_to(Z, (n,)), dtype=np.float64)
    out = np.empty((6, n))
    st = np.empty(n, dtype=np.int32)
    lib().orc_props_at_Z(tb.ref, n, _ptr(T), _ptr(p), _ptr(Y), _ptr(Z), _ptr(out), _ptr(st))
    return out, st


def diagnose(sp, T, p, Y, **kw):
    """Per-cell diagnostics (list of dicts) plus outputs and status."""
    tb = sp if isinstance(sp, Table) else Table(sp, **kw)
    T, p, Y = _soa(T, p, Y, tb.n)
    n = T.size
    out = np.empty((6, n))
    st = np.empty(n, dtype=np.int32)
    diags = (Diag * n)()
    lib().orc_diagnose(tb.ref, n, _ptr(T), _ptr(p), _ptr(Y), _ptr(out), _ptr(st), ctypes.cast(diags, ctypes.c_void_p))
    res = []
    for d in diags:
        res.append({f: (list(getattr(d, f)) if f == "roots" else getattr(d, f)) for f, _ in Diag._fields_})
    return out, st, res


def T_from_h(sp, hstar, p, Y, Tguess, max_iter: int = 60, rtol: float = 1e-13, threads: int = 0, **kw):
    tb = sp if isinstance(sp, Table) else Table(sp, **kw)
    hstar = np.ascontiguousarray(hstar, dtype=np.float64)
    n = hstar.size
    p = np.ascontiguousarray(np.broadcast_to(p, hstar.shape), dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(tb.n, n)
    Tg = np.ascontiguousarray(np.broadcast_to(Tguess, hstar.shape), dtype=np.float64)
    Tout = np.empty(n)
    st = np.empty(n, dtype=np.int32)
    it = np.empty(n, dtype=np.int32)
    lib().orc_T_from_h(tb.ref, n, _ptr(hstar), _ptr(p), _ptr(Y), _ptr(Tg), _ptr(Tout), _ptr(st), _ptr(it),
                       int(max_iter), float(rtol), int(threads))
    return Tout, st, it


class Corr(ctypes.Structure):
    _fields_ = [("n_Tr", ctypes.c_int32), ("n_pr", ctypes.c_int32), ("Tr", ctypes.c_void_p),
                ("pr", ctypes.c_void_p), ("f", ctypes.c_void_p)]


def species_props(sp, T, p, Y, corr=None, threads: int = 0, **kw):
    """(hk_RT[N, n], Dk[N, n], status[n]): the per-species standard-state
    enthalpies h_k/(R T) and mixture-averaged diffusion coefficients [m^2/s].
    ``corr`` = (Tr axis, pr axis, f[len(Tr), len(pr)]) is the high-pressure
    correction table (None: no correction)."""
    tb = sp if isinstance(sp, Table) else Table(sp, **kw)
    T, p, Y = _soa(T, p, Y, tb.n)
    n = T.size
    hk = np.empty((tb.n, n))
    Dk = np.empty((tb.n, n))
    st = np.empty(n, dtype=np.int32)
    cref = None
    if corr is not None:
        Tr, pr, f = (np.ascontiguousarray(a, dtype=np.float64) for a in corr)
        assert f.shape == (Tr.size, pr.size)
        keep = (Tr, pr, f)
        cs = Corr(Tr.size, pr.size, _ptr(Tr), _ptr(pr), _ptr(f))
        cref = ctypes.byref(cs)
    lib().orc_species_props(tb.ref, cref, n, _ptr(T), _ptr(p), _ptr(Y), _ptr(hk), _ptr(Dk), _ptr(st), int(threads))
    if corr is not None:
        del keep
    return hk, Dk, st


def bilger_z(sp, atoms, Y_fuel, Y_ox, Y):
    """Bilger's mixture fraction of n cells (Y [N, n]); atoms [N, 3] = C, H, O."""
    W = np.ascontiguousarray(sp.W, dtype=np.float64)
    N = W.size
    a = np.ascontiguousarray(atoms, dtype=np.int32).reshape(N, 3)
    yf = np.ascontiguousarray(Y_fuel, dtype=np.float64)
    yo = np.ascontiguousarray(Y_ox, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(N, -1)
    Z = np.empty(Y.shape[1])
    lib().orc_bilger_z(N, _ptr(a), _ptr(W), _ptr(yf), _ptr(yo), Y.shape[1], _ptr(Y), _ptr(Z))
    return Z


def neufeld_omega_d(Ts):
    return lib().orc_neufeld_omega_d(float(Ts))


def cubic_real_roots(c2, c1, c0):
    r = np.zeros(3)
    n = lib().orc_cubic_real_roots(float(c2), float(c1), float(c0), _ptr(r))
    return r[:n]


def pr_constants(printed: bool = False):
    a = np.zeros(1)
    b = np.zeros(1)
    lib().orc_pr_constants(int(printed), _ptr(a), _ptr(b))
    return float(a[0]), float(b[0])


def gres(Z, A, B):
    return lib().orc_pr_gres(float(Z), float(A), float(B))


def max_threads() -> int:
    return int(lib().orc_max_threads())
