"""The library's FP64 exp, expm1, log and log1p (csrc/pr_math64.cuh, Tang's
table-driven methods) against references in extended precision (numpy's
long double: 64-bit significands on x86, 113-bit on aarch64): within 1.5
units in the last place over the argument ranges of the property paths (and
beyond), as CUDA's own functions are."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FN = {"exp": 0, "expm1": 1, "log": 2, "log1p": 3}


def _ref(name, x):
    f = {"exp": np.exp, "expm1": np.expm1, "log": np.log, "log1p": np.log1p}[name]
    return f(x.astype(np.longdouble))


def _ulps(y, ref):
    """|y - ref| in units of the last place of ref rounded to double."""
    rd = ref.astype(np.float64)
    ulp = np.where(rd != 0, np.spacing(np.abs(rd)), np.finfo(float).tiny)
    return (np.abs(y.astype(np.longdouble) - ref) / ulp).astype(np.float64)


def _args(name, rng):
    if name == "exp":
        return np.concatenate([rng.uniform(-500, 500, 4000), rng.uniform(-2, 2, 3000), rng.uniform(-1e-8, 1e-8, 500),
                               [0.0, 1e-300, -1e-300, 0.5 * np.log(2) / 64, 700.0, -700.0]])
    if name == "expm1":
        return np.concatenate([rng.uniform(-6, 6, 4000), rng.uniform(-0.02, 0.02, 3000),
                               np.exp(rng.uniform(-60, -1, 1000)), -np.exp(rng.uniform(-60, -1, 1000)), [0.0]])
    if name == "log":
        return np.concatenate([np.exp(rng.uniform(-690, 690, 4000)), rng.uniform(0.9, 1.1, 3000),
                               1.0 + np.exp(rng.uniform(-50, -5, 500)), 1.0 - np.exp(rng.uniform(-50, -5, 500)),
                               [1.0, 2.0, 0.5, 1.0 - 2.0 ** -53, 1e-300, 1e300]])
    return np.concatenate([np.exp(rng.uniform(-60, 5, 5000)), -np.exp(rng.uniform(-60, np.log(0.5), 2000)),
                           [0.0, 1e-320, 100.0]])


@pytest.mark.parametrize("name", ["exp", "expm1", "log", "log1p"])
def test_math64_within_one_ulp(prlib, cuda, name):
    import torch
    from paper_2312_04830_gb300 import binding
    L = binding.lib()
    L.pr_eval_math.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.pr_eval_math.restype = ctypes.c_int
    x = _args(name, np.random.default_rng(FN[name] + 7))
    xd = torch.as_tensor(x, dtype=torch.float64, device=cuda)
    ours, cud = torch.empty_like(xd), torch.empty_like(xd)
    s = torch.cuda.current_stream().cuda_stream
    assert L.pr_eval_math(FN[name], x.size, xd.data_ptr(), ours.data_ptr(), s) == 0
    assert L.pr_eval_math(FN[name] + 4, x.size, xd.data_ptr(), cud.data_ptr(), s) == 0
    torch.cuda.synchronize()
    ref = _ref(name, x)
    u_ours = _ulps(ours.cpu().numpy(), ref)
    u_cuda = _ulps(cud.cpu().numpy(), ref)
    print(f"{name}: max ulp ours {u_ours.max():.3f} (mean {u_ours.mean():.3f}), CUDA {u_cuda.max():.3f}")
    # within 1.5 ulp: CUDA's own expm1 and log1p reach 1.05 and 1.46 ulp on these arguments
    assert u_ours.max() <= 1.5, x[np.argmax(u_ours)]
