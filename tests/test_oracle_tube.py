"""Pins of the oracle's tube centre and width (Sec. V-A, Eqs. 18b, 20-21), CPU only."""
import itertools

import numpy as np

from oracle import tube
from paper_2607_01203_b300 import inputs


def _traj(w, b):
    sl = slice(b * w.N, (b + 1) * w.N)
    return w.Phi[b].astype(np.float64), w.c[sl].astype(np.float64), w.r[sl].astype(np.float64)


def test_first_step_closed_form():
    """k = 1: Phi^x_{1,0} = I, so the state part is c_0 +- (|e| + r_0); the input part is K_1 c_0 +-
    |K_1| (|e| + r_0)."""
    w = inputs.tube(n_traj=1, N=4, n_x=5, n_u=2)
    Phi, c, r = _traj(w, 0)
    mu, sigma = tube.tube(Phi, w.N, c, r, w.e.astype(np.float64))
    K1 = Phi[tube.block_index(1, 0)][w.n_x:]
    assert np.allclose(mu[1, :w.n_x], c[0], rtol=0, atol=1e-15)
    assert np.allclose(sigma[1, :w.n_x], np.abs(w.e) + r[0], rtol=1e-14)
    assert np.allclose(mu[1, w.n_x:], K1 @ c[0], rtol=1e-14)
    assert np.allclose(sigma[1, w.n_x:], np.abs(K1) @ (np.abs(w.e) + r[0]), rtol=1e-14)
    assert np.all(mu[0] == 0) and np.all(sigma[0] == 0)


def test_width_is_attained_at_a_vertex():
    """Brute force on a tiny loop: over every vertex xi_j in {-1, 1}^{2 n_x} of every disturbance up to
    k, the extreme of each row of sum_j Phi_{k,j} (c_j + Ebar_j xi_j) equals mu_k +- sigma_k (the row-wise
    l1 norm is the support function of the zonotope in the row's direction)."""
    w = inputs.tube(n_traj=1, N=3, n_x=2, n_u=1)
    Phi, c, r = _traj(w, 0)
    mu, sigma = tube.tube(Phi, w.N, c, r, w.e.astype(np.float64))
    for k in range(1, w.N + 1):
        Eb = [tube.ebar(w.e.astype(np.float64), r[j]) for j in range(k)]
        best_hi = np.full(w.n_x + w.n_u, -np.inf)
        best_lo = np.full(w.n_x + w.n_u, np.inf)
        for bits in itertools.product((-1.0, 1.0), repeat=4 * k):
            xi = np.array(bits).reshape(k, 4)
            v = sum(Phi[tube.block_index(k, j)] @ (c[j] + Eb[j] @ xi[j]) for j in range(k))
            best_hi = np.maximum(best_hi, v)
            best_lo = np.minimum(best_lo, v)
        assert np.allclose(best_hi, mu[k] + sigma[k], rtol=1e-13, atol=1e-17)
        assert np.allclose(best_lo, mu[k] - sigma[k], rtol=1e-13, atol=1e-17)


def test_closed_loop_simulation_stays_in_the_tube():
    """The responses are those of the loop e_{k+1} = A_k e_k + B_k u_k + d_k, u_k = K_k e_k, e_0 = 0: every
    simulated error with d_j in the zonotope c_j + Ebar_j E lies in the box, and the sign vertex of a
    row's support reaches its bound."""
    w = inputs.tube(n_traj=2, N=12, n_x=6, n_u=3)
    rng = np.random.default_rng(70)
    for b in range(w.n_traj):
        _, c, r = _traj(w, b)
        Phi = w.Phi64[b]   # the responses of that loop before their rounding to FP32
        mu, sigma = tube.tube(Phi, w.N, c, r, w.e.astype(np.float64))
        Eb = [tube.ebar(w.e.astype(np.float64), r[j]) for j in range(w.N)]
        for trial in range(200):
            xi = rng.uniform(-1, 1, (w.N, 2 * w.n_x))
            if trial < 2 * w.n_x:   # also push every disturbance to the vertex that maximises one state row
                row = trial % w.n_x
                xi = np.array([np.sign((Phi[tube.block_index(w.N, j)] @ Eb[j])[row]) for j in range(w.N)])
            e = np.zeros(w.n_x)
            for k in range(w.N + 1):
                u = w.K[b, k] @ e
                z = np.concatenate([e, u])
                assert np.all(np.abs(z - mu[k]) <= sigma[k] * (1 + 1e-12) + 1e-15), (b, k)
                if k == w.N and trial < 2 * w.n_x:
                    assert abs(z[row] - (mu[k][row] + sigma[k][row])) <= 1e-12 * sigma[k][row]
                if k < w.N:
                    e = (w.A[b, k] + w.B[b, k] @ w.K[b, k]) @ e + c[k] + Eb[k] @ xi[k]


def test_dense_disturbance_scaling_and_per_step_matrices():
    """Ebar_j = [E(z_j) R_j] with a dense, per-timestep E(z_j): the width equals the row sums of the
    absolute explicit product, and splitting it as |Phi E| 1 + |Phi| r holds (R_j is diagonal)."""
    w = inputs.tube(n_traj=1, N=5, n_x=4, n_u=2)
    Phi, c, r = _traj(w, 0)
    rng = np.random.default_rng(71)
    Es = [rng.normal(size=(w.n_x, 3)) * 1e-2 for _ in range(w.N)]
    mu, sigma = tube.tube(Phi, w.N, c, r, Es)
    for k in range(1, w.N + 1):
        s = sum(np.abs(Phi[tube.block_index(k, j)] @ Es[j]).sum(1) + np.abs(Phi[tube.block_index(k, j)]) @ r[j]
                for j in range(k))
        assert np.allclose(sigma[k], s, rtol=1e-13)
