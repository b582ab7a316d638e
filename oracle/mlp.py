"""Float64 NumPy surrogate MLP -- TEST INFRASTRUCTURE ONLY (see oracle/__init__).

The paper's surrogate (Sec. 4.1) is a multilayer perceptron with GeLU
activations trained with PyTorch; the configuration here has 11 inputs
(log T, p, Y_1..Y_9), four hidden layers of 512 and 6 outputs
(log rho, Z, h, log cp, log mu, log lambda), inputs and outputs standardised.

Definitions (plain, unfused):
  * GeLU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2   (exact form, "erf")
    or Hendrycks & Gimpel's tanh form ("tanh"), Phi(z) replaced by
    (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) / 2; the paper names GeLU
    without saying which, the tensor-core path computes the tanh form
  * layer l:  z_l = W_l h_{l-1} + b_l,  h_l = GeLU(z_l)  (linear last layer)
  * loss on standardised targets s:  L = mean_{b, j} (yhat_bj - s_bj)^2
    (the targets are logarithms or scaled values, so squared errors are
    relative errors: the relative-MSE loss), or the paper's L1 norm (Sec. 4.3)
    L = mean_{b, j} |yhat_bj - s_bj|, whose gradient takes sign(0) = 0
  * backward: the chain rule, layer by layer
  * Adam (Kingma & Ba): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    p <- p - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)

Pins (tests/test_oracle_mlp.py): gradients against central finite
differences of the loss, GeLU identities, Adam's first step.
"""
from __future__ import annotations

import math

import numpy as np

SQRT2 = math.sqrt(2.0)


def _erf(x):
    # numpy has no erf; vectorise math.erf (exact to double rounding)
    return np.vectorize(math.erf, otypes=[np.float64])(x)


TANH_C = math.sqrt(2.0 / math.pi)
TANH_A = 0.044715


def gelu(z, form="erf"):
    if form == "tanh":
        return 0.5 * z * (1.0 + np.tanh(TANH_C * (z + TANH_A * z ** 3)))
    return 0.5 * z * (1.0 + _erf(z / SQRT2))


def gelu_grad(z, form="erf"):
    """d/dz GeLU(z): Phi(z) + z phi(z) for the exact form; for the tanh
    form, with u = c (z + a z^3) and t = tanh u,
    (1 + t) / 2 + z (1 - t^2) c (1 + 3 a z^2) / 2."""
    if form == "tanh":
        t = np.tanh(TANH_C * (z + TANH_A * z ** 3))
        return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * TANH_C * (1.0 + 3.0 * TANH_A * z * z)
    return 0.5 * (1.0 + _erf(z / SQRT2)) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(sizes, seed=0):
    """PyTorch-Linear-style U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    rng = np.random.default_rng(seed)
    params = []
    for fin, fout in zip(sizes[:-1], sizes[1:]):
        bound = 1.0 / math.sqrt(fin)
        params.append((rng.uniform(-bound, bound, (fout, fin)), rng.uniform(-bound, bound, fout)))
    return params


def forward(params, X, form="erf"):
    """X [B, n_in] -> (yhat [B, n_out], cache of (z_l, h_l))."""
    h = np.asarray(X, dtype=np.float64)
    cache = [(None, h)]
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        h = gelu(z, form) if li + 1 < len(params) else z
        cache.append((z, h))
    return h, cache


# ------------------------------------------------ BF16 storage (inference)
def bf16(x):
    """Round to the nearest BF16 number (ties to even), via float32: the
    storage format of the tensor-core path's weights and activations."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16_storage(params, X, form="tanh"):
    """The forward pass with the values rounded where the tensor-core path
    stores them in BF16: every weight, the inputs as a pair hi = bf16(x),
    lo = bf16(x - hi) (both multiplied by the same weight) and every hidden
    activation after GeLU; the arithmetic in float64.  Returns (yhat,
    cache of (z_l, h_l before rounding, h_l stored))."""
    x = np.asarray(X, dtype=np.float64)
    hi = bf16(x)
    h = hi + bf16(x - hi)
    cache = [(None, x, h)]
    for li, (W, b) in enumerate(params):
        z = h @ bf16(W).T + b
        if li + 1 < len(params):
            g = gelu(z, form)
            h = bf16(g)
            cache.append((z, g, h))
        else:
            h = z
            cache.append((z, z, z))
    return h, cache


def loss(yhat, s, kind="mse"):
    if kind == "l1":
        return float(np.mean(np.abs(yhat - s)))
    return float(np.mean((yhat - s) ** 2))


def backward(params, cache, yhat, s, form="erf", kind="mse"):
    """Gradients of `loss` (of the same kind) w.r.t. every (W_l, b_l)."""
    B, J = yhat.shape
    dz = (np.sign(yhat - s) if kind == "l1" else 2.0 * (yhat - s)) / (B * J)
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        h_prev = cache[li][1]
        grads[li] = (dz.T @ h_prev, dz.sum(axis=0))
        if li > 0:
            dh = dz @ W
            dz = dh * gelu_grad(cache[li][0], form)
    return grads


def adam_step(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; state = {"t": int, "m": [[mW, mb], ...], "v": [...]} (created if empty)."""
    if not state:
        state.update(t=0, m=[[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
                     v=[[np.zeros_like(W), np.zeros_like(b)] for W, b in params])
    state["t"] += 1
    t = state["t"]
    new = []
    for li, (pl, gl) in enumerate(zip(params, grads)):
        out = []
        for k in range(2):
            g = gl[k]
            state["m"][li][k] = b1 * state["m"][li][k] + (1 - b1) * g
            state["v"][li][k] = b2 * state["v"][li][k] + (1 - b2) * g * g
            mh = state["m"][li][k] / (1 - b1 ** t)
            vh = state["v"][li][k] / (1 - b2 ** t)
            out.append(pl[k] - lr * mh / (np.sqrt(vh) + eps))
        new.append(tuple(out))
    return new


# ------------------------------------------------------------- transforms
def input_features(T, p, Y):
    """[log T, p, Y_1..Y_N] per cell, [B, N+2]."""
    return np.column_stack([np.log(T), p, np.asarray(Y).T])


def output_targets(props, h_ig):
    """props [6, B] = rho, Z, h, cp, mu, lambda and the ideal-gas enthalpy
    h_ig [B] of the same states -> [log rho, Z, h - h_ig, log cp, log mu,
    log lambda], [B, 6].  The network learns the enthalpy departure; the
    ideal-gas part (NASA-7, exact) is added back to its output."""
    rho, Z, h, cp, mu, lam = props
    return np.column_stack([np.log(rho), Z, h - h_ig, np.log(cp), np.log(mu), np.log(lam)])


def targets_to_props(q, h_ig):
    """Inverse of output_targets: [B, 6] -> [6, B]."""
    return np.vstack([np.exp(q[:, 0]), q[:, 1], q[:, 2] + h_ig, np.exp(q[:, 3]), np.exp(q[:, 4]),
                      np.exp(q[:, 5])])
