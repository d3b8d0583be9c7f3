"""Pins of the learned-operator network oracle (FP64): finite-difference
gradients, GELU closed forms, Adam against its definition on a quadratic."""
import math

import numpy as np

import workloads as W
from oracle import mlp


def _net(seed=3):
    return mlp.unflatten(W.mlp_init(seed))


def test_param_count_and_packing():
    v = W.mlp_init(2)
    assert v.size == 64 + 64 + 4096 + 64 + 4096 + 64 + 26 * 64 + 26
    assert np.array_equal(mlp.flatten(mlp.unflatten(v)), v)


def test_gelu_closed_forms():
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu(np.array(10.0)) - 10.0) < 1e-12
    assert abs(mlp.gelu(np.array(-10.0))) < 1e-12
    # gelu(1) = 0.5 (1 + erf(1/sqrt 2)) = Phi(1) = 0.841344746...
    assert abs(mlp.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    a = np.linspace(-4, 4, 81)
    fd = (mlp.gelu(a + 1e-6) - mlp.gelu(a - 1e-6)) / 2e-6
    assert np.max(np.abs(fd - mlp.gelu_grad(a))) < 1e-8


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    p = _net()
    x = rng.uniform(0, 1, 7)
    t = rng.normal(0, 0.3, (7, 26))
    y, cache = mlp.forward(p, x)
    g = mlp.flatten(mlp.backward(p, cache, y, t))
    v = mlp.flatten(p)
    idx = rng.choice(v.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(v)
        e[i] = 1e-6
        lp = mlp.loss(mlp.forward(mlp.unflatten(v + e), x)[0], t)
        lm = mlp.loss(mlp.forward(mlp.unflatten(v - e), x)[0], t)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_linear_special_case():
    # W2 = W3 = 0: h2 = gelu(b2), h3 = gelu(b3) independent of x, so y = W4 gelu(b3) + b4.
    p = _net()
    p["W2"][:] = 0
    p["W3"][:] = 0
    p["b3"][:] = np.linspace(-1, 1, 64)
    y, _ = mlp.forward(p, np.array([0.1, 0.9]))
    ref = p["W4"] @ mlp.gelu(p["b3"]) + p["b4"]
    assert np.allclose(y, ref[None, :], rtol=0, atol=1e-13)


def test_adam_first_step_is_sign_step():
    # After one step from zero moments, the bias-corrected update is lr * g / (|g| + eps).
    v = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    v1, m, s = mlp.adam_step(v, g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(v1, v - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
