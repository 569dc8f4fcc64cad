"""Sampled true linearization errors (Eq. 9c) for soundness checks, FP64.

A sound enclosure [r_lo, r_hi] over a set must contain r(alpha) = f(alpha) - f(alpha~) - [A B](alpha - alpha~)
for every alpha in the set, where [A B] is the linearization the bound was computed for. Points are drawn
from the box interior, its vertices and its faces (one coordinate free, the rest at a bound), and from a
zonotope's generator combinations (interior and sign vertices).
"""
from __future__ import annotations

import numpy as np


def box_points(lo, hi, count: int, rng: np.random.Generator) -> np.ndarray:
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    n = lo.shape[0]
    k1 = count // 3
    k2 = count // 3
    k3 = count - k1 - k2
    U = rng.uniform(size=(k1, n))
    interior = lo + U * (hi - lo)
    V = rng.integers(0, 2, size=(k2, n)).astype(np.float64)
    vertices = lo + V * (hi - lo)
    F = rng.integers(0, 2, size=(k3, n)).astype(np.float64)
    free = rng.integers(0, n, size=k3)
    F[np.arange(k3), free] = rng.uniform(size=k3)
    faces = lo + F * (hi - lo)
    return np.concatenate([interior, vertices, faces])


def zonotope_points(center, G, count: int, rng: np.random.Generator) -> np.ndarray:
    G = np.asarray(G, np.float64)
    p = G.shape[1]
    half = count // 2
    xi_in = rng.uniform(-1.0, 1.0, size=(half, p))
    xi_v = rng.choice([-1.0, 1.0], size=(count - half, p))
    # the vertices that attain each row's hull extreme are always included
    rows = rng.integers(0, G.shape[0], size=min(64, count - half))
    for t, r in enumerate(rows):
        xi_v[t] = np.sign(G[r]) * (1 if t % 2 == 0 else -1)
    xi = np.concatenate([xi_in, xi_v])
    return np.asarray(center, np.float64)[None, :] + xi @ G.T


def remainders(f_batch, nominal, lin, points) -> np.ndarray:
    """r(alpha) for every row of ``points`` [P, n]; ``f_batch`` maps [P, n] -> [P, n_x]."""
    a = np.asarray(nominal, np.float64)
    P = np.asarray(points, np.float64)
    f0 = f_batch(a[None, :])[0]
    return f_batch(P) - f0[None, :] - (P - a[None, :]) @ np.asarray(lin, np.float64).T


def mlp_f_batch(Ws, bs, act: str, residual: bool = True):
    Ws = [np.asarray(W, np.float64) for W in Ws]
    bs = [np.asarray(b, np.float64) for b in bs]
    n_x = Ws[-1].shape[0]

    def f(P):
        h = P
        for i, (W, b) in enumerate(zip(Ws, bs)):
            h = h @ W.T + b
            if i + 1 < len(Ws):
                h = np.maximum(h, 0.0) if act == "relu" else np.tanh(h)
        return h + P[:, :n_x] if residual else h
    return f
