"""ctypes binding of libprgb300.so (argument marshalling only).

Every function here checks tensor dtypes, devices and shapes, then passes raw
device pointers and the current CUDA stream to the C ABI declared in
``include/prgb300.h``.  All arithmetic runs in the library's kernels; there is
no CPU path: if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libprgb300.so")

PR_FP64, PR_FP32, PR_MIXED = 0, 1, 2
PRECISIONS = {"fp64": PR_FP64, "fp32": PR_FP32, "mixed": PR_MIXED}
PR_FLAG_PRINTED_CONSTANTS = 1
PR_FLAG_TRANSPORT_XAVG = 2
OUTPUTS = ("rho", "Z", "h", "cp", "mu", "lambda")

CELL_STATUS = {0: "ok", 1: "newton_maxit", 2: "h_out_of_range", 3: "no_root", 4: "bad_input", 5: "ambiguous"}

_lock = threading.Lock()
_lib = None


class PrError(RuntimeError):
    pass


class _SpeciesTable(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("flags", ctypes.c_int32)] + [
        (f, ctypes.c_void_p) for f in ("W", "Tc", "pc", "omega", "Vc", "dipole", "kappa",
                                        "nasa_lo", "nasa_hi", "T_mid", "kij")]


def lib():
    """Load libprgb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise PrError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2312_04830_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            L.pr_create.argtypes = [ctypes.POINTER(_SpeciesTable), ctypes.POINTER(vp)]
            L.pr_create.restype = i32
            L.pr_destroy.argtypes = [vp]
            L.pr_destroy.restype = None
            L.pr_props.argtypes = [vp, i32, i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            L.pr_props.restype = i32
            L.pr_T_from_h.argtypes = [vp, i32, i64, vp, vp, vp, i64, vp, vp, vp, vp, i32, d, vp]
            L.pr_T_from_h.restype = i32
            L.pr_last_error.argtypes = []
            L.pr_last_error.restype = ctypes.c_char_p
            L.pr_version.argtypes = []
            L.pr_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def check(status: int, what: str):
    if status != 0:
        msg = lib().pr_last_error().decode(errors="replace")
        raise PrError(f"{what} failed with status {status}: {msg}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_of(prec: int):
    import torch
    return torch.float64 if prec == PR_FP64 else torch.float32


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


class PropertyContext:
    """A species table resident on the current CUDA device (pr_create)."""

    def __init__(self, species, printed_constants: bool = False, transport_xavg: bool = False):
        self._keep = {}
        arr = lambda name, a: self._keep.setdefault(name, np.ascontiguousarray(a, dtype=np.float64))
        n = int(species.n)
        kij = getattr(species, "kij", None)
        t = _SpeciesTable()
        t.n_species = n
        t.flags = (PR_FLAG_PRINTED_CONSTANTS if printed_constants else 0) | \
                  (PR_FLAG_TRANSPORT_XAVG if transport_xavg else 0)
        for f in ("W", "Tc", "pc", "omega", "Vc", "dipole", "kappa", "T_mid"):
            setattr(t, f, arr(f, getattr(species, f)).ctypes.data)
        t.nasa_lo = arr("nasa_lo", species.nasa_lo).ctypes.data
        t.nasa_hi = arr("nasa_hi", species.nasa_hi).ctypes.data
        t.kij = arr("kij", kij).ctypes.data if kij is not None else None
        self.n_species = n
        h = ctypes.c_void_p()
        check(lib().pr_create(ctypes.byref(t), ctypes.byref(h)), "pr_create")
        self.handle = h
        self._keep.clear()

    def close(self):
        if getattr(self, "handle", None):
            lib().pr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- helpers
    def _cells(self, prec, T, p, Y):
        import torch
        dt = _dtype_of(prec)
        for name, t in (("T", T), ("p", p), ("Y", Y)):
            if not isinstance(t, torch.Tensor) or not t.is_cuda:
                raise PrError(f"{name} must be a CUDA tensor")
            if t.dtype != dt:
                raise PrError(f"{name} must be {dt} for this precision, got {t.dtype}")
        n = T.numel()
        if T.dim() != 1 or p.shape != T.shape or not T.is_contiguous() or not p.is_contiguous():
            raise PrError("T and p must be contiguous 1-D tensors of equal length")
        if Y.dim() != 2 or Y.shape[0] != self.n_species or Y.shape[1] != n or Y.stride(1) != 1:
            raise PrError(f"Y must be [{self.n_species}, n] with unit stride along cells")
        return n, Y.stride(0) if n > 0 else max(n, 1)

    # --------------------------------------------------------------- calls
    def props(self, T, p, Y, precision="fp64", out=None, status=None, outputs=OUTPUTS, stream=None):
        """Forward properties; returns (out[6, n] rows rho, Z, h, cp, mu, lambda; status[n])."""
        import torch
        prec = _prec(precision)
        n, ldY = self._cells(prec, T, p, Y)
        if out is None:
            out = torch.empty((6, n), dtype=_dtype_of(prec), device=T.device)
        if status is None:
            status = torch.empty(n, dtype=torch.int32, device=T.device)
        ptrs = [(_ptr(out[q]) if OUTPUTS[q] in outputs else None) for q in range(6)]
        check(lib().pr_props(self.handle, prec, n, _ptr(T), _ptr(p), _ptr(Y), ldY, *ptrs, _ptr(status),
                             _stream(stream)), "pr_props")
        return out, status

    def T_from_h(self, hstar, p, Y, T_guess, precision="fp64", max_iter=60, rtol=1e-13, T_out=None,
                 status=None, iters=None, stream=None):
        """Newton inversion T(h*, p, Y); returns (T, status, iters)."""
        import torch
        prec = _prec(precision)
        n, ldY = self._cells(prec, hstar, p, Y)
        if T_guess.dtype != hstar.dtype or T_guess.shape != hstar.shape or not T_guess.is_contiguous():
            raise PrError("T_guess must match hstar")
        if T_out is None:
            T_out = torch.empty_like(hstar)
        if status is None:
            status = torch.empty(n, dtype=torch.int32, device=hstar.device)
        if iters is None:
            iters = torch.empty(n, dtype=torch.int32, device=hstar.device)
        check(lib().pr_T_from_h(self.handle, prec, n, _ptr(hstar), _ptr(p), _ptr(Y), ldY, _ptr(T_guess),
                                _ptr(T_out), _ptr(status), _ptr(iters), int(max_iter), float(rtol),
                                _stream(stream)), "pr_T_from_h")
        return T_out, status, iters
