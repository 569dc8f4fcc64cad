"""The learned LEB proposer's network in FP64: forward, backward and one Adam step.

The proposer maps (x~_k, u~_k, state radii) to standardised (r_lo, r_hi). It is a ReLU MLP
392 -> 256 -> 256 -> 336 trained with mean-squared error on standardised targets. (It is an addition to
the paper's method, whose bounds it only proposes; the certified bound stays the answer.)

Layout: weights W_i are [out, in], inputs X are [B, in], outputs [B, out].
The proposer's specification fixes its arithmetic to BF16 GEMM operands with FP32 (here FP64)
accumulation; with ``bf16=True`` every matrix-product operand is rounded to BF16 (round to nearest, ties
to even) before the product, as the definition of that precision.
Loss = mean over all B*out entries of (Y - T)^2.
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as FP64."""
    f = np.asarray(x, np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return rounded.view(np.float32).astype(np.float64)


def _op(x, on):
    return bf16(x) if on else np.asarray(x, np.float64)


def forward(params, X, bf16_ops=False):
    Ws, bs = params
    h = np.asarray(X, np.float64)
    cache = [h]
    for i, (W, b) in enumerate(zip(Ws, bs)):
        z = _op(h, bf16_ops) @ _op(W, bf16_ops).T + np.asarray(b, np.float64)
        if i + 1 < len(Ws):
            h = np.maximum(z, 0.0)
        else:
            h = z
        cache.append(z)
    return h, cache


def loss_and_grads(params, X, Tgt, bf16_ops=False):
    Ws, bs = params
    Y, cache = forward(params, X, bf16_ops)
    B, out = Y.shape
    diff = Y - np.asarray(Tgt, np.float64)
    loss = float((diff ** 2).mean())
    g = 2.0 * diff / (B * out)                  # dLoss/dY
    gWs = [None] * len(Ws)
    gbs = [None] * len(Ws)
    for i in range(len(Ws) - 1, -1, -1):
        h_in = cache[0] if i == 0 else np.maximum(cache[i], 0.0)
        gWs[i] = _op(g, bf16_ops).T @ _op(h_in, bf16_ops)
        gbs[i] = g.sum(axis=0)
        if i > 0:
            g = (_op(g, bf16_ops) @ _op(Ws[i], bf16_ops)) * (cache[i] > 0)
    return loss, gWs, gbs


def adam_step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
