"""Pins of the FP64 MLP restatement (oracle/mlp.py): the analytic gradient
against central finite differences of its own loss, and the GELU against its
closed-form limits and derivative."""
import math

import numpy as np

from oracle import mlp


def random_params(rng):
    P = rng.standard_normal(mlp.NPARAM) * 0.3
    P[0:6] = rng.standard_normal(6)
    P[6:12] = rng.uniform(0.5, 2.0, 6)
    P[12], P[13] = 0.3, 1.7
    return P


def test_gelu():
    z = np.linspace(-6, 6, 101)
    g = mlp.gelu(z)
    assert abs(mlp.gelu(np.array([0.0]))[0]) == 0.0
    assert np.allclose(g[z > 5], z[z > 5], rtol=1e-6) and np.allclose(g[z < -5], 0, atol=1e-5)
    h = 1e-5
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_d(z), fd, atol=1e-9)
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 1e-15


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = random_params(rng)
    F = rng.standard_normal((40, 6)) * 2 + 1
    T = rng.standard_normal(40)
    loss, g = mlp.loss_and_grad(P, F, T)
    h = 1e-6
    idx = rng.choice(len(g), 120, replace=False)
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[14 + i] += h
        Pm[14 + i] -= h
        fd = (mlp.loss_and_grad(Pp, F, T)[0] - mlp.loss_and_grad(Pm, F, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
