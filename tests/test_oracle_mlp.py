"""Pins of the float64 MLP oracle (CPU)."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_identities():
    """GeLU(0) = 0; GeLU(-z) = GeLU(z) - z (from Phi(-z) = 1 - Phi(z));
    GeLU(z) -> z for large z and -> 0 for very negative z; Phi(1) from the
    normal table (0.8413447461)."""
    z = np.linspace(-6, 6, 241)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(mlp.gelu(-z), mlp.gelu(z) - z, atol=1e-15)
    assert mlp.gelu(np.array([12.0]))[0] == pytest.approx(12.0, rel=1e-15)
    assert abs(mlp.gelu(np.array([-12.0]))[0]) < 1e-30
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-12)


def test_gelu_tanh_form_against_exact():
    """The tanh form keeps GeLU(0) = 0 and the odd-part identity (tanh is
    odd) and stays within 5e-4 of the exact form everywhere (its largest
    deviation, 4.7e-4, is near |z| = 2.7); a wrong cubic coefficient or
    scale would break that bound."""
    z = np.linspace(-8, 8, 16001)
    t = mlp.gelu(z, "tanh")
    assert mlp.gelu(np.array([0.0]), "tanh")[0] == 0.0
    np.testing.assert_allclose(mlp.gelu(-z, "tanh"), t - z, atol=1e-14)
    dev = np.abs(t - mlp.gelu(z))
    assert dev.max() < 5e-4 and dev.max() > 4e-4
    assert mlp.gelu(np.array([12.0]), "tanh")[0] == pytest.approx(12.0, rel=1e-15)


@pytest.mark.parametrize("form", ["erf", "tanh"])
def test_gelu_grad_matches_finite_difference(form):
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (mlp.gelu(z + h, form) - mlp.gelu(z - h, form)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z, form), fd, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("form,kind", [("erf", "mse"), ("tanh", "mse"), ("tanh", "l1")])
def test_backward_matches_finite_difference(form, kind):
    """Every gradient of a tiny 5-layer net against central differences of
    the loss (FP64, step 1e-6, 1e-5 for L1); for the L1 loss no residual is
    within 1e-3 of its kink, so the step never crosses one."""
    sizes = [11, 7, 6, 5, 4, 6]
    params = mlp.init_params(sizes, seed=3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(9, 11))
    s = rng.normal(size=(9, 6))
    yhat, cache = mlp.forward(params, X, form)
    assert np.abs(yhat - s).min() > 1e-3
    grads = mlp.backward(params, cache, yhat, s, form, kind)
    h = 1e-6 if kind == "mse" else 1e-5   # L1: a larger step keeps round-off (eps L / h) below 1e-10
    for li, (W, b) in enumerate(params):
        for k, P in enumerate((W, b)):
            flat = P.reshape(-1)
            for idx in range(0, flat.size, max(1, flat.size // 7)):
                old = flat[idx]
                flat[idx] = old + h
                lp = mlp.loss(mlp.forward(params, X, form)[0], s, kind)
                flat[idx] = old - h
                lm = mlp.loss(mlp.forward(params, X, form)[0], s, kind)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                g = grads[li][k].reshape(-1)[idx]
                assert g == pytest.approx(fd, rel=1e-6, abs=1e-10), (li, k, idx)


def test_l1_loss_closed_form():
    """The L1 loss is the mean absolute residual; its output gradient is
    sign(residual) / (B J), zero where the residual is zero."""
    yhat = np.array([[1.0, -2.0, 0.5], [0.0, 3.0, -1.0]])
    s = np.array([[0.0, -2.0, 1.5], [1.0, 1.0, -1.0]])
    assert mlp.loss(yhat, s, "l1") == pytest.approx((1 + 0 + 1 + 1 + 2 + 0) / 6)
    params = [(np.eye(3), np.zeros(3))]
    g = mlp.backward(params, [(None, yhat)], yhat, s, "tanh", "l1")
    assert np.allclose(g[0][1], np.array([0.0, 1.0, -1.0]) / 6)


def test_adam_first_step_is_signed_lr():
    """With zero moments, Adam's first update is lr g / (|g| + eps') = lr sign(g)
    up to eps (bias corrections cancel exactly)."""
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -4.0]]), np.array([1e-3]))]
    st = {}
    new = mlp.adam_step(params, grads, st, lr=0.01)
    np.testing.assert_allclose(new[0][0], [[0.99, -1.99]], rtol=1e-7)
    np.testing.assert_allclose(new[0][1], [0.49], rtol=1e-6)
    assert st["t"] == 1


def test_adam_converges_on_quadratic():
    """Brute-force sanity: Adam on a convex quadratic reaches the minimiser."""
    target = np.array([[0.7, -1.3]])
    params = [(np.zeros((1, 2)), np.zeros(1))]
    st = {}
    for _ in range(3000):
        g = [(2 * (params[0][0] - target), 2 * (params[0][1] - 0.2))]
        params = mlp.adam_step(params, g, st, lr=0.01)
    np.testing.assert_allclose(params[0][0], target, atol=1e-3)
    np.testing.assert_allclose(params[0][1], [0.2], atol=1e-3)


def test_output_transform_roundtrip():
    rng = np.random.default_rng(0)
    props = np.vstack([rng.uniform(1, 1000, 5), rng.uniform(0.1, 1.2, 5), rng.uniform(-1e7, 1e7, 5),
                       rng.uniform(1e3, 1e5, 5), rng.uniform(1e-6, 1e-3, 5), rng.uniform(1e-2, 1, 5)])
    h_ig = rng.uniform(-1e7, 1e7, 5)
    q = mlp.output_targets(props, h_ig)
    np.testing.assert_allclose(q[:, 2], props[2] - h_ig, rtol=1e-15)
    np.testing.assert_allclose(mlp.targets_to_props(q, h_ig), props, rtol=1e-14, atol=1e-8)
