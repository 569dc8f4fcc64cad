"""Tube centre and width from the linearization-error bounds (Sec. V-A), plain FP64.

Test infrastructure (the oracle), not part of the product path.

The LEB of timestep j enters the SLS problem through the zonotope map Gamma (Sec. IV-C): its centre
c_j and diagonal radius R_j = diag(r_j) (Eq. 22 with the padding of Sec. V-A). The zonotope of the
exogenous disturbance and the linearization error is c_j + Ebar_j E_{2 n_x} with the generator matrix
Ebar_j = [E(z_j)  R_j] (Eq. 18b). Given the system responses Phi_{k,j} = [Phi^x_{k,j}; Phi^u_{k,j}]
((n_x + n_u) x n_x, j < k), the tube centre and width of timestep k are (Eqs. 20-21)

    h^mu_k    = sum_{j<k} Phi_{k,j} c_j,
    h^sigma_k = sum_{j<k} || Phi_{k,j} Ebar_j ||_{1,r}     (row-wise l1 norm),

and the reachable tube of timestep k lies in the box [h^mu_k - h^sigma_k, h^mu_k + h^sigma_k] around the
nominal (Eq. 19). Written out from the definitions: Ebar_j as an explicit matrix, the products with a
library matmul, the row-wise l1 norm as the sum of absolute values.

Packed layout of the responses (shared with the C ABI): block p = k (k - 1) / 2 + j for 1 <= k <= N,
0 <= j < k, each block (n_x + n_u) x n_x row-major, state rows first; P = N (N + 1) / 2 blocks per
trajectory. Timestep k = 0 has an empty sum (centre and width 0).
"""
from __future__ import annotations

import numpy as np


def block_index(k: int, j: int) -> int:
    """Position of Phi_{k,j} in the packed layout (1 <= k, 0 <= j < k)."""
    assert 0 <= j < k
    return k * (k - 1) // 2 + j


def ebar(E: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Eq. 18b: the generator matrix [E(z_j)  diag(r_j)]; E is n_x x n_e (a vector is read as diag(E))."""
    E = np.asarray(E, np.float64)
    if E.ndim == 1:
        E = np.diag(E)
    return np.concatenate([E, np.diag(np.asarray(r, np.float64))], axis=1)


def tube(Phi: np.ndarray, N: int, c: np.ndarray, r: np.ndarray, E) -> tuple[np.ndarray, np.ndarray]:
    """Eqs. 20-21 for one trajectory.

    Phi: [P, n_x + n_u, n_x] packed responses; c, r: [N, n_x] Gamma-map centres and radii of the
    timesteps 0..N-1; E: one n_x x n_e matrix or a vector (diag), or a list of N of them (E(z_j)).
    Returns (mu, sigma), each [N + 1, n_x + n_u]."""
    Phi = np.asarray(Phi, np.float64)
    rows = Phi.shape[1]
    per_step = isinstance(E, (list, tuple)) or (np.ndim(E) == 3) or (np.ndim(E) == 2 and np.shape(E)[0] == N
                                                                       and np.shape(E)[1] == Phi.shape[2]
                                                                       and N != Phi.shape[2])
    mu = np.zeros((N + 1, rows))
    sigma = np.zeros((N + 1, rows))
    for k in range(1, N + 1):
        for j in range(k):
            Pk = Phi[block_index(k, j)]
            Ej = E[j] if per_step else E
            mu[k] += Pk @ np.asarray(c[j], np.float64)
            sigma[k] += np.abs(Pk @ ebar(Ej, r[j])).sum(axis=1)
    return mu, sigma
