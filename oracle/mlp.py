"""Oracle for the warm-start network (test infrastructure; FP64 numpy).

The plain definition of the MLP the library trains: layers in -> hidden (GELU)
x layers -> out (linear), parameters flat as [W (out x in) row-major, b (out)]
per layer, loss = mean over all outputs of (Y - T)^2, GELU(x) = x/2 (1 +
erf(x / sqrt 2)).  The gradient is written out by the chain rule; a central
finite-difference check pins it in the CPU tests.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special as sp


def layout(dims):
    """(W offset, b offset) of every layer in the flat parameter array."""
    offs = []
    o = 0
    for i in range(len(dims) - 1):
        nw = dims[i] * dims[i + 1]
        offs.append((o, o + nw))
        o += nw + dims[i + 1]
    return offs, o


def unpack(p, dims):
    offs, _ = layout(dims)
    Ws, bs = [], []
    for i, (ow, ob) in enumerate(offs):
        Ws.append(p[ow:ow + dims[i] * dims[i + 1]].reshape(dims[i + 1], dims[i]))
        bs.append(p[ob:ob + dims[i + 1]])
    return Ws, bs


def gelu(x):
    return 0.5 * x * (1.0 + sp.erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + sp.erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(p, dims, X):
    Ws, bs = unpack(np.asarray(p, dtype=np.float64), dims)
    a = np.asarray(X, dtype=np.float64)
    zs, acts = [], [a]
    for i in range(len(Ws)):
        z = a @ Ws[i].T + bs[i]
        zs.append(z)
        a = gelu(z) if i < len(Ws) - 1 else z
        acts.append(a)
    return a, zs, acts


def loss_and_grad(p, dims, X, T):
    Y, zs, acts = forward(p, dims, X)
    T = np.asarray(T, dtype=np.float64)
    n = Y.size
    loss = float(np.sum((Y - T) ** 2) / n)
    Ws, _ = unpack(np.asarray(p, dtype=np.float64), dims)
    offs, total = layout(dims)
    g = np.zeros(total)
    dz = 2.0 * (Y - T) / n
    for i in range(len(Ws) - 1, -1, -1):
        ow, ob = offs[i]
        g[ow:ow + Ws[i].size] = (dz.T @ acts[i]).ravel()
        g[ob:ob + dims[i + 1]] = dz.sum(axis=0)
        if i > 0:
            dz = (dz @ Ws[i]) * gelu_grad(zs[i - 1])
    return loss, g
