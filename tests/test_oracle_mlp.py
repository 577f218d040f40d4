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


# Phi(1) and Phi(-1) of the standard normal distribution (printed in every
# normal table): GELU(1) = 1 * Phi(1), GELU(-1) = -Phi(-1).
PHI_1 = 0.8413447460685429
PHI_M1 = 0.15865525393145707


def hand_network():
    """A network whose output can be worked out by hand: hidden units that
    read nothing sit at z = -40, where GELU is exactly 0 in FP64, and z = 40
    gives GELU exactly 40.  Feature standardisation fm = 1..6, fs = 2."""
    P = np.zeros(mlp.NPARAM)
    P[0:6] = np.arange(1, 7)
    P[6:12] = 2.0
    W1 = np.zeros((mlp.NH, mlp.NF))
    b1 = np.full(mlp.NH, -40.0)
    W2 = np.zeros((mlp.NH, mlp.NH))
    b2 = np.full(mlp.NH, -40.0)
    w3 = np.zeros(mlp.NH)
    # hidden unit 5 of layer 1: z = 10 x_2 + 5 x_4 + 10  (x standardised)
    W1[5, 2], W1[5, 4], b1[5] = 10.0, 5.0, 10.0
    # hidden unit 9 of layer 1: z = x_0 - 1
    W1[9, 0], b1[9] = 1.0, -1.0
    # layer 2 unit 3 reads unit 5: z = h5 / 40 - 0 (so z = 1 when h5 = 40)
    W2[3, 5], b2[3] = 1.0 / 40.0, 0.0
    # layer 2 unit 7 reads unit 9: z = h9 + 0.5
    W2[7, 9], b2[7] = 1.0, 0.5
    w3[3], w3[7], b3 = 2.0, -3.0, 0.25
    P[mlp.OFF_W1:mlp.OFF_B1] = W1.ravel()  # 64 x 6 row-major: W1[i, j] at 6 i + j
    P[mlp.OFF_B1:mlp.OFF_W2] = b1
    P[mlp.OFF_W2:mlp.OFF_B2] = W2.ravel()
    P[mlp.OFF_B2:mlp.OFF_W3] = b2
    P[mlp.OFF_W3:mlp.OFF_B3] = w3
    P[mlp.OFF_B3] = b3
    return P


def test_forward_matches_hand_computation():
    """forward() pinned by outputs worked out by hand from the layer equations
    z1 = W1 (f - fm) / fs + b1, h1 = GELU(z1), z2 = W2 h1 + b2,
    h2 = GELU(z2), out = w3 . h2 + b3 (parameter layout of include/hm.h).
    A swapped standardisation, a dropped bias or a transposed weight layout
    each changes these values."""
    P = hand_network()
    F = np.array([
        [-1.0, 0.0, 7.0, 0.0, 1.0, 0.0],   # x0 = -1, x2 = 2, x4 = -2 -> z1[5] = 20, z1[9] = -2
        [5.0, 0.0, 3.0, 0.0, 5.0, 0.0],    # x0 = 2,  x2 = 0, x4 = 0  -> z1[5] = 10, z1[9] = 1
        [1.0, 0.0, 9.0, 0.0, 9.0, 0.0],    # x0 = 0,  x2 = 3, x4 = 2  -> z1[5] = 50, z1[9] = -1
        [3.0, 0.0, 9.0, 0.0, 5.0, 0.0],    # x0 = 1,  x2 = 3, x4 = 0  -> z1[5] = 40, z1[9] = 0
    ])
    out, (X, Z1, H1, Z2, H2) = mlp.forward(P, F)
    assert np.array_equal(X[:, [0, 2, 4]], [[-1, 2, -2], [2, 0, 0], [0, 3, 2], [1, 3, 0]])
    assert np.array_equal(Z1[:, 5], [20, 10, 50, 40]) and np.array_equal(Z1[:, 9], [-2, 1, -1, 0])
    # units that read nothing sit at z = -40: exactly 0 after the GELU
    assert not H1[:, [i for i in range(mlp.NH) if i not in (5, 9)]].any()
    assert not H2[:, [i for i in range(mlp.NH) if i not in (3, 7)]].any()
    # GELU(z) = z Phi(z): exactly z at z >= 10 in FP64, Phi(+-1) from the normal table
    assert np.array_equal(H1[:, 5], [20, 10, 50, 40])
    assert abs(H1[1, 9] - PHI_1) < 1e-16 and abs(H1[2, 9] + PHI_M1) < 1e-16 and H1[3, 9] == 0
    # layer 2: z2[3] = h1[5] / 40, z2[7] = h1[9] + 0.5
    assert np.array_equal(Z2[:, 3], [0.5, 0.25, 1.25, 1.0])
    assert abs(Z2[1, 7] - (PHI_1 + 0.5)) < 1e-15 and abs(Z2[2, 7] - (0.5 - PHI_M1)) < 1e-15
    assert Z2[3, 7] == 0.5
    # row 3: out = 2 GELU(1) - 3 GELU(0.5) + 0.25 with GELU(0.5) = 0.5 Phi(0.5),
    # Phi(0.5) = 0.6914624612740131 (normal table)
    assert abs(out[3] - (2.0 * PHI_1 - 1.5 * 0.6914624612740131 + 0.25)) < 1e-15
