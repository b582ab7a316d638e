"""Per-sample bound on the difference between the tensor-core surrogate's
standardised outputs and the float64 oracle MLP with BF16 storage
(oracle.mlp.forward_bf16_storage), from a first-order error analysis.

Storage rounding is the same on both sides, so what remains is local error
the GPU adds at each hidden activation: its pre-activation z differs by the
FP32 accumulation (at most gamma_K(FP32) sum_i |w_i h_i|, K the fan-in plus
the bias), its GeLU by the hardware tanh (tanh.approx.f32; relative error
below 2^-10.98 per the PTX ISA, taken as 2^-10 here), and where the two
values fall on either side of a BF16 rounding boundary the stored activations
differ by one BF16 ulp.  With J_l = d y / d h_l (the oracle network's
Jacobian, rounding taken as the identity), the output error is at most
sum_l |J_l| e_l, e_l the bound of the local error at layer l; the first layer's
hi/lo input pair is exact to about 2^-16 and its FP32 standardisation error is
included the same way.
"""
import numpy as np

from oracle import mlp as omlp

U32 = 2.0 ** -24             # FP32 unit roundoff
EPS_TANH = 2.0 ** -10        # hardware tanh, relative (bounded by 2^-10.98)
GELU_D = 1.13                # max |d GeLU / d z| of the tanh form


def _gelu_grad(z):
    return omlp.gelu_grad(z, "tanh")


def _ulp_bf16(h):
    """One BF16 ulp at h (2^(e-8) for |h| in [2^(e-1), 2^e))."""
    _, e = np.frexp(h)
    return np.ldexp(1.0, e - 8)


def output_error_bound(params, s_in, in_err):
    """Bound [B, n_out] on |s_gpu - s_oracle_bf16| per sample and output;
    in_err [B, n_in]: bound on the GPU's standardised inputs' distance from
    s_in (its FP32 features and standardisation)."""
    yhat, cache = omlp.forward_bf16_storage(params, s_in, "tanh")
    L = len(params)
    n_out = params[-1][0].shape[0]
    B = s_in.shape[0]
    # local error bounds e_l [B, width] at each stored activation h_l, l = 1..L-1
    e = []
    x0 = cache[0][2]
    for li in range(L - 1):
        W, b = params[li]
        Wb = omlp.bf16(W)
        h_prev = cache[li][2]
        z, g, hs = cache[li + 1]
        acc = (np.abs(h_prev) @ np.abs(Wb).T + np.abs(b)) * (W.shape[1] + 1) * U32 / (1 - (W.shape[1] + 1) * U32)
        if li == 0:   # the inputs: FP32 standardisation, then the hi/lo pair (exact to 2^-17)
            acc += (in_err + 2.0 ** -17 * np.abs(s_in)) @ np.abs(Wb).T
        dg = GELU_D * acc + 0.5 * np.abs(z) * EPS_TANH + 2 * U32 * np.abs(g)
        ulp = _ulp_bf16(np.maximum(np.abs(hs), np.abs(g)))
        near = np.abs(g - hs) >= 0.5 * ulp - dg       # the GPU's value may round to the neighbour
        e.append(dg + near * 2 * ulp)
    # Jacobians d y_j / d h_l by backward passes through the oracle network
    bound = np.zeros((B, n_out))
    for j in range(n_out):
        v = np.zeros((B, n_out))
        v[:, j] = 1.0
        g = v @ omlp.bf16(params[-1][0])                # d y_j / d h_{L-1}
        for li in range(L - 2, -1, -1):
            bound[:, j] += np.sum(np.abs(g) * e[li], axis=1)
            if li > 0:
                z = cache[li + 1][0]
                g = (g * _gelu_grad(z)) @ omlp.bf16(params[li][0])
        # the output layer's own FP32 accumulation
        Wo, bo = params[-1]
        bound[:, j] += (np.abs(cache[L - 1][2]) @ np.abs(omlp.bf16(Wo[j])) + abs(bo[j])) * \
            (Wo.shape[1] + 1) * U32
    return yhat, bound
