"""ORACLE -- test infrastructure only.  fp64 forward and backward of the job
cost network (12 -> 64 -> 64 -> 1, ReLU), written as the chain rule by hand,
and its training by Adam (Kingma and Ba, "Adam: A Method for Stochastic
Optimization", ICLR 2015, Algorithm 1) on full batches.

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


# Adam's default hyper-parameters (Kingma and Ba, Algorithm 1)
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def adam_step(p, g, m1, m2, t: int, lr: float):
    """One Adam update at step t >= 1, returning (p, m1, m2):
    m1 <- beta1 m1 + (1 - beta1) g;  m2 <- beta2 m2 + (1 - beta2) g^2;
    p <- p - lr * (m1 / (1 - beta1^t)) / (sqrt(m2 / (1 - beta2^t)) + eps)."""
    p = np.asarray(p, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m1 = BETA1 * np.asarray(m1, dtype=np.float64) + (1.0 - BETA1) * g
    m2 = BETA2 * np.asarray(m2, dtype=np.float64) + (1.0 - BETA2) * g * g
    mhat = m1 / (1.0 - BETA1 ** t)
    vhat = m2 / (1.0 - BETA2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + EPS), m1, m2


def train(p, x, y, steps: int, lr: float):
    """``steps`` full-batch Adam steps on the mean squared error from p.
    Returns the parameters, the loss after the last step and the gradient
    of every step (steps x NPARAMS)."""
    p = np.asarray(p, dtype=np.float64).copy()
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    grads = []
    for t in range(1, steps + 1):
        _, g = loss_and_grad(p, x, y)
        grads.append(g)
        p, m1, m2 = adam_step(p, g, m1, m2, t, lr)
    loss, _ = loss_and_grad(p, x, y)
    return p, loss, np.array(grads).reshape(-1, NPARAMS)
