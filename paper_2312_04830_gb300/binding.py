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
PR_FLAG_NEWTON_FP64_ONLY = 4
OUTPUTS = ("rho", "Z", "h", "cp", "mu", "lambda")
OUTPUTS_EXT = OUTPUTS + ("psi", "alpha")

CELL_STATUS = {0: "ok", 1: "newton_maxit", 2: "h_out_of_range", 3: "no_root", 4: "bad_input", 5: "ambiguous"}

_lock = threading.Lock()
_lib = None


class PrError(RuntimeError):
    pass


PEAK_KINDS = {"fp64_fma": 0, "fp32_fma": 1, "mufu_ex2": 2, "fp64_exp": 3, "fp64_log": 4, "fp64_div": 5,
              "fp64_sqrt": 6, "fp64_cbrt": 7}


def measure_peak(kind: str) -> float:
    """Measured throughput of one arithmetic pipe on the current device:
    flops/s for 'fp64_fma' and 'fp32_fma', exp2/s for 'mufu_ex2', calls/s of
    CUDA's FP64 exp, log, division, square root and cube root for 'fp64_exp',
    'fp64_log', 'fp64_div', 'fp64_sqrt', 'fp64_cbrt'."""
    v = ctypes.c_double(0.0)
    check(lib().pr_measure_peak(PEAK_KINDS[kind], ctypes.byref(v)), "pr_measure_peak")
    return v.value


class _DiffCorr(ctypes.Structure):
    _fields_ = [("n_Tr", ctypes.c_int32), ("n_pr", ctypes.c_int32), ("Tr", ctypes.c_void_p),
                ("pr", ctypes.c_void_p), ("f", ctypes.c_void_p)]


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
            L.pr_props_ext.argtypes = [vp, i32, i64, vp, vp, vp, i64] + [vp] * 8 + [vp, vp]
            L.pr_props_ext.restype = i32
            L.pr_props.restype = i32
            L.pr_species_props.argtypes = [vp, i32, i64, vp, vp, vp, i64, vp, vp, i64, vp, vp]
            L.pr_species_props.restype = i32
            L.pr_set_diffusion_correction.argtypes = [vp, vp]
            L.pr_set_diffusion_correction.restype = i32
            L.pr_set_bilger.argtypes = [vp, vp, vp, vp]
            L.pr_set_bilger.restype = i32
            L.pr_bilger_z.argtypes = [vp, i32, i64, vp, i64, vp, vp]
            L.pr_bilger_z.restype = i32
            L.pr_measure_peak.argtypes = [i32, vp]
            L.pr_measure_peak.restype = i32
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

    def __init__(self, species, printed_constants: bool = False, transport_xavg: bool = False,
                 newton_fp64_only: bool = False):
        self._keep = {}
        arr = lambda name, a: self._keep.setdefault(name, np.ascontiguousarray(a, dtype=np.float64))
        n = int(species.n)
        kij = getattr(species, "kij", None)
        t = _SpeciesTable()
        t.n_species = n
        t.flags = (PR_FLAG_PRINTED_CONSTANTS if printed_constants else 0) | \
                  (PR_FLAG_TRANSPORT_XAVG if transport_xavg else 0) | \
                  (PR_FLAG_NEWTON_FP64_ONLY if newton_fp64_only else 0)
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

    def props_ext(self, T, p, Y, precision="fp64", out=None, status=None, outputs=OUTPUTS_EXT, stream=None):
        """pr_props_ext; returns (out[8, n] rows rho, Z, h, cp, mu, lambda, psi, alpha; status[n])."""
        import torch
        prec = _prec(precision)
        n, ldY = self._cells(prec, T, p, Y)
        if out is None:
            out = torch.empty((8, n), dtype=_dtype_of(prec), device=T.device)
        if status is None:
            status = torch.empty(n, dtype=torch.int32, device=T.device)
        ptrs = [(_ptr(out[q]) if OUTPUTS_EXT[q] in outputs else None) for q in range(8)]
        check(lib().pr_props_ext(self.handle, prec, n, _ptr(T), _ptr(p), _ptr(Y), ldY, *ptrs, _ptr(status),
                                 _stream(stream)), "pr_props_ext")
        return out, status

    def species_props(self, T, p, Y, precision="fp64", hk=True, Dk=True, status=None, stream=None):
        """pr_species_props; returns (hk_RT[N, n] or None, Dk[N, n] or None, status[n]):
        per-species h_k/(R T) and mixture-averaged diffusion coefficients [m^2/s].
        hk / Dk: True (allocate), False (skip) or a [N, n] tensor to fill."""
        import torch
        prec = _prec(precision)
        n, ldY = self._cells(prec, T, p, Y)

        def mk(o):
            if o is True:
                return torch.empty((self.n_species, n), dtype=_dtype_of(prec), device=T.device)
            if o is False or o is None:
                return None
            if o.dtype != _dtype_of(prec) or tuple(o.shape) != (self.n_species, n) or not o.is_contiguous():
                raise PrError(f"species output must be a contiguous [{self.n_species}, {n}] {_dtype_of(prec)} tensor")
            return o
        hk_t, dk_t = mk(hk), mk(Dk)
        if status is None:
            status = torch.empty(n, dtype=torch.int32, device=T.device)
        check(lib().pr_species_props(self.handle, prec, n, _ptr(T), _ptr(p), _ptr(Y), ldY, _ptr(hk_t), _ptr(dk_t),
                                     n, _ptr(status), _stream(stream)), "pr_species_props")
        return hk_t, dk_t, status

    def set_bilger(self, atoms, Y_fuel, Y_ox):
        """Element table ([N, 3] C, H, O atoms) and the fuel / oxidiser streams of
        Bilger's mixture fraction."""
        a = np.ascontiguousarray(atoms, dtype=np.int32).reshape(self.n_species, 3)
        yf = np.ascontiguousarray(Y_fuel, dtype=np.float64)
        yo = np.ascontiguousarray(Y_ox, dtype=np.float64)
        if yf.size != self.n_species or yo.size != self.n_species:
            raise PrError("stream compositions must have one entry per species")
        check(lib().pr_set_bilger(self.handle, a.ctypes.data, yf.ctypes.data, yo.ctypes.data), "pr_set_bilger")

    def bilger_z(self, Y, precision="fp64", out=None, stream=None):
        """Bilger's mixture fraction of the cells of Y [N, n]."""
        import torch
        prec = _prec(precision)
        if not isinstance(Y, torch.Tensor) or not Y.is_cuda or Y.dtype != _dtype_of(prec) or Y.dim() != 2 \
                or Y.shape[0] != self.n_species or Y.stride(1) != 1:
            raise PrError(f"Y must be a CUDA [{self.n_species}, n] {_dtype_of(prec)} tensor with unit cell stride")
        n = Y.shape[1]
        if out is None:
            out = torch.empty(n, dtype=Y.dtype, device=Y.device)
        check(lib().pr_bilger_z(self.handle, prec, n, _ptr(Y), Y.stride(0), _ptr(out), _stream(stream)),
              "pr_bilger_z")
        return out

    def set_diffusion_correction(self, Tr=None, pr=None, f=None):
        """High-pressure factor f(T_r, p_r) of the binary diffusion coefficients
        as a table (Tr rows, pr columns); no arguments remove it."""
        if Tr is None:
            check(lib().pr_set_diffusion_correction(self.handle, None), "pr_set_diffusion_correction")
            return
        Tr, pr, f = (np.ascontiguousarray(a, dtype=np.float64) for a in (Tr, pr, f))
        if f.shape != (Tr.size, pr.size):
            raise PrError("f must be [len(Tr), len(pr)]")
        c = _DiffCorr(Tr.size, pr.size, Tr.ctypes.data, pr.ctypes.data, f.ctypes.data)
        check(lib().pr_set_diffusion_correction(self.handle, ctypes.byref(c)), "pr_set_diffusion_correction")

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


# ------------------------------------------------------------------ surrogate
class _SgConfig(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("hidden_layers", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("infer_chunk", ctypes.c_int32)]


SG_NORM_FLOATS = 84
SG_OPT_FUSED_INFER = 1
SG_OPT_MODE, SG_MODE_FORWARD, SG_MODE_INVERSE, SG_MODE_BILGER = 2, 0, 1, 2
SG_OPT_WAIT_LIMIT_KCYCLES, SG_OPT_TEST_STALL = 3, 4
SG_OPT_LOSS, SG_LOSS_REL_MSE, SG_LOSS_L1 = 5, 0, 1
SG_OPT_CONFIDENCE_PPM = 6
SG_OPT_OUTPUTS, SG_OUT_PROPS, SG_OUT_DK, SG_OUT_HK, SG_OUT_SINGLE = 7, 0, 1, 2, 3
# the single-property networks, in the inverse model's output order
SINGLE_OUTPUTS = ("T", "rho", "psi", "mu", "alpha", "cp")
SG_OPT_TRANSPORT_CONFIDENCE_PPM = 8
SG_OPT_TIME_MLP = 9
N_RAW, N_IN, N_OUT = 11, 13, 6   # raw inputs (T, p, Y_1..Y_9), network inputs, outputs


def _sg_lib():
    L = lib()
    if not getattr(L, "_sg_ready", False):
        vp, i64, i32, f32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_uint64
        L.surrogate_create.argtypes = [vp, ctypes.POINTER(_SgConfig), u64, ctypes.POINTER(vp)]
        L.surrogate_create.restype = i32
        L.surrogate_destroy.argtypes = [vp]
        L.surrogate_destroy.restype = None
        L.surrogate_num_params.argtypes = [vp]
        L.surrogate_num_params.restype = i64
        for fn in ("surrogate_get_params", "surrogate_set_params"):
            getattr(L, fn).argtypes = [vp, vp, i64]
            getattr(L, fn).restype = i32
        for fn in ("surrogate_get_normalization", "surrogate_set_normalization"):
            getattr(L, fn).argtypes = [vp, vp]
            getattr(L, fn).restype = i32
        L.surrogate_fit_normalization.argtypes = [vp, i64, vp, i64, vp, i64, vp]
        L.surrogate_fit_normalization.restype = i32
        L.surrogate_train_step.argtypes = [vp, i64, i64, vp, i64, vp, i64, u64, f32, vp, vp]
        L.surrogate_train_step.restype = i32
        L.surrogate_loss_grad.argtypes = [vp, i64, vp, i64, vp, i64, vp, vp, vp]
        L.surrogate_loss_grad.restype = i32
        L.surrogate_infer.argtypes = [vp, i64, vp, vp, vp, i64, vp, i64, vp, vp]
        L.surrogate_infer.restype = i32
        L.surrogate_set_option.argtypes = [vp, i32, i32]
        L.surrogate_set_option.restype = i32
        L.surrogate_get_option.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int)]
        L.surrogate_get_option.restype = i32
        L.surrogate_set_boxcox.argtypes = [vp, ctypes.c_double, ctypes.c_double]
        L.surrogate_set_boxcox.restype = i32
        L.surrogate_sync_status.argtypes = [vp]
        L.surrogate_sync_status.restype = i32
        L.surrogate_mlp_time.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        L.surrogate_mlp_time.restype = i32
        L.surrogate_save.argtypes = [vp, ctypes.c_char_p]
        L.surrogate_save.restype = i32
        L.surrogate_load.argtypes = [vp, ctypes.c_char_p]
        L.surrogate_load.restype = i32
        L.mlp_gemm_bf16.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp]
        L.mlp_gemm_bf16.restype = i32
        L._sg_ready = True
    return L


class Surrogate:
    """The surrogate MLP bound to a PropertyContext (its PR fallback)."""

    def __init__(self, ctx: PropertyContext, width=512, hidden_layers=4, max_batch=65536, infer_chunk=1 << 20,
                 seed=1):
        L = _sg_lib()
        self.ctx = ctx
        cfg = _SgConfig(width, hidden_layers, max_batch, infer_chunk)
        h = ctypes.c_void_p()
        check(L.surrogate_create(ctx.handle, ctypes.byref(cfg), ctypes.c_uint64(seed), ctypes.byref(h)),
              "surrogate_create")
        self.handle = h
        self.width, self.hidden_layers, self.max_batch = width, hidden_layers, max_batch

    def set_mode(self, mode: str):
        """'forward' (T, p, Y -> rho, Z, h, cp, mu, lambda), 'inverse' (h*, p, Y
        -> T, rho, psi, mu, alpha, cp) or 'bilger' (as inverse, the network
        seeing h*, p and Bilger's mixture fraction of Y; needs the context's
        set_bilger); set before fitting and training."""
        v = {"forward": SG_MODE_FORWARD, "inverse": SG_MODE_INVERSE, "bilger": SG_MODE_BILGER}[mode]
        check(_sg_lib().surrogate_set_option(self.handle, SG_OPT_MODE, v), "surrogate_set_option")
        self.mode = mode

    def set_boxcox(self, lam: float, shift: float = 1e-3):
        """Box-Cox parameters of Bilger's mixture fraction (bilger mode)."""
        check(_sg_lib().surrogate_set_boxcox(self.handle, float(lam), float(shift)), "surrogate_set_boxcox")

    def set_fused_infer(self, on):
        """All layers of an inference chunk in one launch ('resident', the
        default for widths 256 and 512: CTA pairs that keep each 256-row
        block's activations in shared memory through all layers; True:
        activation rings in L2, 128 x 256 tiles, one CTA each; 'pair': the
        same with 256 x 256 tiles on CTA pairs), or one launch per layer
        (False); 'pingpong': CTA pairs whose activations alternate between
        tensor memory and shared memory from layer to layer."""
        v = {"pair": 2, "resident": 3, "pingpong": 4}.get(on, None) if isinstance(on, str) else int(bool(on))
        if v is None:
            raise ValueError(f"unknown fused-inference kind {on!r}")
        check(_sg_lib().surrogate_set_option(self.handle, SG_OPT_FUSED_INFER, v), "surrogate_set_option")

    def get_option(self, option: int) -> int:
        """Current value of a model option (SG_OPT_*); for SG_OPT_FUSED_INFER
        the kernel the next inference runs: 0 per layer, 1 single CTAs, 2
        CTA pairs, 3 resident activations, 4 alternating activations."""
        v = ctypes.c_int(0)
        check(_sg_lib().surrogate_get_option(self.handle, int(option), ctypes.byref(v)), "surrogate_get_option")
        return v.value

    @property
    def fused_kind(self) -> str:
        """'pingpong', 'resident', 'pair', 'single' or 'per-layer': the inference kernel in use."""
        return {0: "per-layer", 1: "single", 2: "pair", 3: "resident", 4: "pingpong"}[self.get_option(SG_OPT_FUSED_INFER)]

    def set_loss(self, kind: str):
        """Training loss: 'mse' (relative MSE on the standardised targets, the
        default) or 'l1' (the paper's L1 norm)."""
        v = {"mse": SG_LOSS_REL_MSE, "l1": SG_LOSS_L1}[kind]
        check(_sg_lib().surrogate_set_option(self.handle, SG_OPT_LOSS, v), "surrogate_set_option")
        self.loss_kind = kind

    def set_confidence(self, tol: float):
        """Forward model: cells whose predicted rho and Z disagree with the
        equation of state (|rho Z R T / (p W) - 1| > tol) take the FP64
        fallback; 0 turns the test off."""
        check(_sg_lib().surrogate_set_option(self.handle, SG_OPT_CONFIDENCE_PPM, int(round(tol * 1e6))),
              "surrogate_set_option")

    def set_transport_confidence(self, tol: float):
        """Property models: cells whose predicted mu or lambda differ by more
        than tol (relative) from Chung's correlation evaluated at the
        network's own density (and temperature, for the inverse models) take
        the FP64 fallback; 0 turns the test off."""
        check(_sg_lib().surrogate_set_option(self.handle, SG_OPT_TRANSPORT_CONFIDENCE_PPM, int(round(tol * 1e6))),
              "surrogate_set_option")

    def set_wait_limit(self, kcycles: int):
        """Limit, in thousands of SM clock cycles, of every bounded wait in the
        fused inference kernel; 0 restores the default (4e9 cycles)."""
        check(_sg_lib().surrogate_set_option(self.handle, SG_OPT_WAIT_LIMIT_KCYCLES, int(kcycles)),
              "surrogate_set_option")

    def set_test_stall(self, on: bool):
        """Test hook: make one dependency of the fused kernel unreachable, so
        that its bounded wait runs out and sync_status raises."""
        check(_sg_lib().surrogate_set_option(self.handle, SG_OPT_TEST_STALL, int(bool(on))), "surrogate_set_option")

    def close(self):
        if getattr(self, "handle", None):
            _sg_lib().surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        return int(_sg_lib().surrogate_num_params(self.handle))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.num_params, dtype=np.float32)
        check(_sg_lib().surrogate_get_params(self.handle, a.ctypes.data, a.size), "surrogate_get_params")
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        check(_sg_lib().surrogate_set_params(self.handle, a.ctypes.data, a.size), "surrogate_set_params")

    def get_normalization(self) -> np.ndarray:
        a = np.empty(SG_NORM_FLOATS, dtype=np.float32)
        check(_sg_lib().surrogate_get_normalization(self.handle, a.ctypes.data), "surrogate_get_normalization")
        return a

    def set_normalization(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        assert a.size == SG_NORM_FLOATS
        check(_sg_lib().surrogate_set_normalization(self.handle, a.ctypes.data), "surrogate_set_normalization")

    @property
    def n_out(self) -> int:
        return getattr(self, "_n_out", N_OUT)

    def set_outputs(self, kind: str):
        """'props' (the mode's six outputs), 'dk' (the 9 mixture-averaged
        diffusion coefficients), 'hk' (the 9 standard-state h_k / (R T)), or
        one of 'T', 'rho', 'psi', 'mu', 'alpha', 'cp' (a dedicated network for
        that property alone); all but 'props' need the inverse or Bilger mode.
        Re-initialises the weights."""
        if kind in SINGLE_OUTPUTS:
            v, n = SG_OUT_SINGLE + SINGLE_OUTPUTS.index(kind), 1
        else:
            v = {"props": SG_OUT_PROPS, "dk": SG_OUT_DK, "hk": SG_OUT_HK}[kind]
            n = N_OUT if v == SG_OUT_PROPS else 9
        check(_sg_lib().surrogate_set_option(self.handle, SG_OPT_OUTPUTS, v), "surrogate_set_option")
        self._n_out = n
        self.single_output = kind if kind in SINGLE_OUTPUTS else None

    def _pool(self, x, y):
        import torch
        for nm, t, rows in (("x", x, N_RAW), ("y", y, self.n_out)):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
                raise PrError(f"{nm} must be a float32 CUDA tensor")
            if t.dim() != 2 or t.shape[0] != rows or t.stride(1) != 1:
                raise PrError(f"{nm} must be [{rows}, n] with unit stride along rows")
        if x.shape[1] != y.shape[1]:
            raise PrError("x and y must have the same number of rows")
        return x.shape[1], x.stride(0), y.stride(0)

    def fit_normalization(self, x, y, stream=None):
        n, ldx, ldy = self._pool(x, y)
        check(_sg_lib().surrogate_fit_normalization(self.handle, n, _ptr(x), ldx, _ptr(y), ldy, _stream(stream)),
              "surrogate_fit_normalization")

    def train_step(self, x, y, batch, lr, sample_seed=0, loss_out=None, stream=None):
        n, ldx, ldy = self._pool(x, y)
        check(_sg_lib().surrogate_train_step(self.handle, batch, n, _ptr(x), ldx, _ptr(y), ldy,
                                             ctypes.c_uint64(sample_seed), ctypes.c_float(lr), _ptr(loss_out),
                                             _stream(stream)), "surrogate_train_step")

    def loss_grad(self, x, y, batch, stream=None):
        import torch
        n, ldx, ldy = self._pool(x, y)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        grad = torch.empty(self.num_params, dtype=torch.float32, device=x.device)
        check(_sg_lib().surrogate_loss_grad(self.handle, batch, _ptr(x), ldx, _ptr(y), ldy, _ptr(loss), _ptr(grad),
                                            _stream(stream)), "surrogate_loss_grad")
        return loss, grad

    def infer(self, T, p, Y, out=None, used_fallback=None, stream=None):
        import torch
        n, ldY = self.ctx._cells(PR_FP32, T, p, Y)
        if out is None:
            out = torch.empty((self.n_out, n), dtype=torch.float32, device=T.device)
        if used_fallback is None:
            used_fallback = torch.empty(n, dtype=torch.uint8, device=T.device)
        check(_sg_lib().surrogate_infer(self.handle, n, _ptr(T), _ptr(p), _ptr(Y), ldY, _ptr(out), out.stride(0),
                                        _ptr(used_fallback), _stream(stream)), "surrogate_infer")
        return out, used_fallback

    def sync_status(self):
        check(_sg_lib().surrogate_sync_status(self.handle), "surrogate_sync_status")

    def set_time_mlp(self, on: bool):
        """Record CUDA events around the MLP launch of every inference chunk
        from now on (restarting the count), or stop."""
        check(_sg_lib().surrogate_set_option(self.handle, SG_OPT_TIME_MLP, int(bool(on))), "surrogate_set_option")

    def mlp_time(self):
        """(milliseconds, launches) of the MLP launches recorded since
        set_time_mlp(True) or the last call; restarts the count."""
        ms, nl = ctypes.c_double(0.0), ctypes.c_int64(0)
        check(_sg_lib().surrogate_mlp_time(self.handle, ctypes.byref(ms), ctypes.byref(nl)), "surrogate_mlp_time")
        return ms.value, nl.value

    def save(self, path):
        check(_sg_lib().surrogate_save(self.handle, str(path).encode()), "surrogate_save")

    def load(self, path):
        check(_sg_lib().surrogate_load(self.handle, str(path).encode()), "surrogate_load")


def gemm_bf16(A, B, D=None, err=None, stream=None):
    """D = A @ B^T on the tensor cores (A [M, K], B [N, K] bfloat16 CUDA tensors)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if D is None:
        D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=A.device)
    check(_sg_lib().mlp_gemm_bf16(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(D), D.stride(0),
                                  _ptr(err), _stream(stream)), "mlp_gemm_bf16")
    return D, err
