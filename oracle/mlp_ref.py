"""Double-precision CPU reference of the per-round scheduler MLP -- TEST
INFRASTRUCTURE ONLY (only tests/, smoke() and bench.py's CPU-baseline leg use
the oracle package).

The network has no counterpart in the paper; it is the 12 -> 32 -> 32 -> 3
ReLU classifier that picks the AC-4, AC-6 or AC-3 kernel for the next round.
Parameter layout (TRIM_MLP_NPARAMS = 1571 floats):
    W1[32][12] b1[32] W2[32][32] b2[32] W3[3][32] b3[3]
Loss: mean softmax cross-entropy over the rows. Adam: Kingma & Ba (2015).

Written from the definitions: z1 = W1 x + b1, h1 = max(z1, 0), z2 = W2 h1 + b2,
h2 = max(z2, 0), z3 = W3 h2 + b3, p = softmax(z3), L = mean(-log p[y]); the
backward pass is the chain rule of these expressions.
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 12, 32, 3
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
         ("W3", (NOUT, NH)), ("b3", (NOUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).reshape(-1) for name, _ in SIZES])


def forward(theta, X):
    """Logits (N, 3) and the intermediate values."""
    P = unpack(theta)
    X = np.asarray(X, np.float64)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ P["W3"].T + P["b3"]
    return z3, (X, z1, h1, z2, h2)


def loss(theta, X, y) -> float:
    z3, _ = forward(theta, X)
    z = z3 - z3.max(axis=1, keepdims=True)
    logp = z - np.log(np.exp(z).sum(axis=1, keepdims=True))
    y = np.asarray(y, np.int64)
    return float(-logp[np.arange(len(y)), y].mean())


def loss_grad(theta, X, y):
    """(mean cross-entropy, gradient w.r.t. theta) by the chain rule."""
    P = unpack(theta)
    z3, (X, z1, h1, z2, h2) = forward(theta, X)
    N = X.shape[0]
    y = np.asarray(y, np.int64)
    z = z3 - z3.max(axis=1, keepdims=True)
    e = np.exp(z)
    p = e / e.sum(axis=1, keepdims=True)
    L = float(-np.log(p[np.arange(N), y]).mean())
    d3 = p.copy()
    d3[np.arange(N), y] -= 1.0
    d3 /= N
    g = {"W3": d3.T @ h2, "b3": d3.sum(axis=0)}
    dh2 = d3 @ P["W3"]
    d2 = dh2 * (z2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    dh1 = d2 @ P["W2"]
    d1 = dh1 * (z1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return L, pack(g)


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def finite_difference_grad(theta, X, y, h=1e-6, idx=None):
    """Central differences of the loss (for checking loss_grad)."""
    theta = np.asarray(theta, np.float64)
    idx = range(theta.size) if idx is None else idx
    g = np.zeros(theta.size)
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        g[i] = (loss(tp, X, y) - loss(tm, X, y)) / (2 * h)
    return g
