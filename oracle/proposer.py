"""The learned LEB proposer's network in FP64: forward, backward and one Adam step.

The proposer maps (x~_k, u~_k, state radii) to standardised (r_lo, r_hi). It is a ReLU MLP
392 -> 256 -> 256 -> 336 trained with mean-squared error on standardised targets. (It is an addition to
the paper's method, whose bounds it only proposes; the certified bound stays the answer.)

Layout: weights W_i are [out, in], inputs X are [B, in], outputs [B, out].
Loss = mean over all B*out entries of (Y - T)^2.
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np


def forward(params, X):
    Ws, bs = params
    h = np.asarray(X, np.float64)
    cache = [h]
    for i, (W, b) in enumerate(zip(Ws, bs)):
        z = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        if i + 1 < len(Ws):
            h = np.maximum(z, 0.0)
        else:
            h = z
        cache.append(z)
    return h, cache


def loss_and_grads(params, X, Tgt):
    Ws, bs = params
    Y, cache = forward(params, X)
    B, out = Y.shape
    diff = Y - np.asarray(Tgt, np.float64)
    loss = float((diff ** 2).mean())
    g = 2.0 * diff / (B * out)                  # dLoss/dY
    gWs = [None] * len(Ws)
    gbs = [None] * len(Ws)
    for i in range(len(Ws) - 1, -1, -1):
        h_in = cache[0] if i == 0 else np.maximum(cache[i], 0.0)
        gWs[i] = g.T @ h_in
        gbs[i] = g.sum(axis=0)
        if i > 0:
            g = (g @ np.asarray(Ws[i], np.float64)) * (cache[i] > 0)
    return loss, gWs, gbs


def adam_step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
