"""ORACLE -- test infrastructure only.  fp64 forward and backward of the job
cost network (12 -> 64 -> 64 -> 1, ReLU), written as the chain rule by hand.

Parameter vector layout: W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3.
Loss: mean squared error of the prediction against the target.
"""
from __future__ import annotations

import numpy as np

F, H = 12, 64
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[k:k + n].reshape(shape)
        k += n
    return out


def forward(p, x):
    w = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    pred = h2 @ w["w3"] + w["b3"][0]
    return pred, (x, z1, h1, z2, h2)


def loss_and_grad(p, x, y):
    """Mean squared error and its gradient with respect to every parameter."""
    w = unpack(p)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    pred, (x, z1, h1, z2, h2) = forward(p, x)
    err = pred - y
    loss = float(np.mean(err * err))
    d3 = 2.0 * err / n                       # dL/dpred
    g_w3 = h2.T @ d3
    g_b3 = np.array([d3.sum()])
    d2 = np.outer(d3, w["w3"]) * (z2 > 0)   # dL/dz2
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ w["W2"]) * (z1 > 0)          # dL/dz1
    g_W1 = d1.T @ x
    g_b1 = d1.sum(axis=0)
    grad = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, g_b3])
    return loss, grad
