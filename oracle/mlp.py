"""FP64 numpy restatement of the rank-predictor MLP (test infrastructure only).

Network 6 -> 64 -> 64 -> 1 with the exact GELU g(z) = z Phi(z), on features
standardised by the mean/deviation stored in the parameter block, loss = mean
squared error of the standardised target.  Forward and backward are written
out layer by layer (chain rule), no library autodiff.  Parameter layout: see
include/hm.h (HM_RANK_MODEL_PARAMS).
"""
import math

import numpy as np

NF, NH = 6, 64
OFF_W1 = 14
OFF_B1 = OFF_W1 + NH * NF
OFF_W2 = OFF_B1 + NH
OFF_B2 = OFF_W2 + NH * NH
OFF_W3 = OFF_B2 + NH
OFF_B3 = OFF_W3 + NH
NPARAM = OFF_B3 + 1

_erf = np.vectorize(math.erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_d(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    return dict(fm=P[0:6], fs=P[6:12], tm=P[12], ts=P[13],
                W1=P[OFF_W1:OFF_B1].reshape(NH, NF), b1=P[OFF_B1:OFF_W2],
                W2=P[OFF_W2:OFF_B2].reshape(NH, NH), b2=P[OFF_B2:OFF_W3],
                w3=P[OFF_W3:OFF_B3], b3=P[OFF_B3])


def forward(P, F):
    p = unpack(P)
    X = (np.asarray(F, np.float64) - p["fm"]) / p["fs"]
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = gelu(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = gelu(Z2)
    out = H2 @ p["w3"] + p["b3"]
    return out, (X, Z1, H1, Z2, H2)


def loss_and_grad(P, F, T):
    """Mean squared error of the standardised target and its gradient with
    respect to the trainable parameters (P[14:])."""
    p = unpack(P)
    out, (X, Z1, H1, Z2, H2) = forward(P, F)
    Y = (np.asarray(T, np.float64) - p["tm"]) / p["ts"]
    B = len(Y)
    r = out - Y
    loss = np.mean(r * r)
    dout = 2.0 * r / B
    g_w3 = H2.T @ dout
    g_b3 = dout.sum()
    dZ2 = np.outer(dout, p["w3"]) * gelu_d(Z2)
    g_W2 = dZ2.T @ H1
    g_b2 = dZ2.sum(0)
    dZ1 = (dZ2 @ p["W2"]) * gelu_d(Z1)
    g_W1 = dZ1.T @ X
    g_b1 = dZ1.sum(0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g
