"""Pins of the FP64 CPU MLP used to check the surrogate's CUDA training kernels:
its analytic gradient against central finite differences, GELU against its definition."""
import math

import numpy as np

from oracle import mlp


def test_gelu_and_its_derivative():
    x = np.linspace(-5, 5, 101)
    ref = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in x])
    np.testing.assert_allclose(mlp.gelu(x), ref, rtol=1e-14, atol=1e-15)
    d = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + d) - mlp.gelu(x - d)) / (2 * d),
                               rtol=1e-8, atol=1e-9)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_par = sum(a * b + b for a, b in mlp.SIZES)
    p = rng.normal(0, 0.2, n_par)
    x = rng.normal(0, 1, (7, 6))
    t = rng.normal(0, 1, (7, 3))
    y, cache = mlp.forward(p, x)
    dy, _ = mlp.mse_grad(y, t)
    g = mlp.backward(p, cache, dy)
    idx = rng.choice(n_par, 60, replace=False)
    for j in idx:
        e = np.zeros(n_par)
        e[j] = 1e-6
        lp = mlp.mse_grad(mlp.forward(p + e, x)[0], t)[1]
        lm = mlp.mse_grad(mlp.forward(p - e, x)[0], t)[1]
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(fd)), j


def test_adam_first_step_is_signed_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.1, 0.0])
    p1, m, v = mlp.adam(p, g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(p1[:2], p[:2] - 0.01 * np.sign(g[:2]), rtol=1e-6)
    assert p1[2] == p[2]
