"""Analytic dynamics of App. A in FP64: model, Jacobian (Eq. 8), Hessian entries for Thm. 1.

Planar quadrotor (App. A, "Planar Quadrotor"), forward Euler with step dt:

    state  (p_x, p_y, phi, v_x, v_y, omega),  input (u_1, u_2),  S = u_1 + u_2
    p_x+   = p_x + dt v_x
    p_y+   = p_y + dt v_y
    phi+   = phi + dt omega
    v_x+   = v_x + dt ( -(S/m) sin(phi) + a^spring_x )
    v_y+   = v_y + dt (  (S/m) cos(phi) - g + a^spring_y )
    omega+ = omega + dt (arm/I)(u_2 - u_1)

The chain stacks ``n_quads`` such quadrotors, states first then inputs
(x = (xi_1..xi_n), u = (u_1..u_n), as in App. A "Coupled 3D Quadrotor"), and couples neighbours'
positions with linear springs of stiffness k: a^spring_{x,i} = (k/m) sum_{j in nbr(i)} (p_{x,j} - p_{x,i}),
free ends (an end quadrotor has one spring). With one quadrotor and k = 0 this is the planar quadrotor.

Coordinates of alpha = [x; u] are 0-based here; the path order of Thm. 1 is this natural order.
"""
from __future__ import annotations

import math
import numpy as np


class QuadChain:
    def __init__(self, n_quads: int, mass: float, inertia: float, arm: float, g: float, dt: float,
                 spring_k: float = 0.0, **_):
        self.nq = int(n_quads)
        self.m, self.I, self.arm, self.g, self.dt, self.k = mass, inertia, arm, g, dt, spring_k
        self.n_x = 6 * self.nq
        self.n_u = 2 * self.nq
        self.n = self.n_x + self.n_u

    # index helpers --------------------------------------------------------------------------
    def ix(self, i: int, s: int) -> int:
        """alpha index of state component s (0..5) of quadrotor i."""
        return 6 * i + s

    def iu(self, i: int, r: int) -> int:
        """alpha index of input r (0, 1) of quadrotor i."""
        return self.n_x + 2 * i + r

    def neighbours(self, i: int):
        return [j for j in (i - 1, i + 1) if 0 <= j < self.nq] if self.k != 0.0 else []

    # model -------------------------------------------------------------------------------------
    def f(self, alpha: np.ndarray) -> np.ndarray:
        a = np.asarray(alpha, np.float64)
        out = np.empty(self.n_x)
        dt, m = self.dt, self.m
        for i in range(self.nq):
            px, py, phi, vx, vy, om = (a[self.ix(i, s)] for s in range(6))
            u1, u2 = a[self.iu(i, 0)], a[self.iu(i, 1)]
            S = u1 + u2
            sx = sum(a[self.ix(j, 0)] - px for j in self.neighbours(i))
            sy = sum(a[self.ix(j, 1)] - py for j in self.neighbours(i))
            out[self.ix(i, 0)] = px + dt * vx
            out[self.ix(i, 1)] = py + dt * vy
            out[self.ix(i, 2)] = phi + dt * om
            out[self.ix(i, 3)] = vx + dt * (-(S / m) * math.sin(phi) + (self.k / m) * sx)
            out[self.ix(i, 4)] = vy + dt * ((S / m) * math.cos(phi) - self.g + (self.k / m) * sy)
            out[self.ix(i, 5)] = om + dt * (self.arm / self.I) * (u2 - u1)
        return out

    def f_batch(self, A: np.ndarray) -> np.ndarray:
        """f for many points at once: A [P, n] -> [P, n_x] (same equations, vectorised)."""
        A = np.asarray(A, np.float64)
        out = np.empty((A.shape[0], self.n_x))
        dt, m = self.dt, self.m
        for i in range(self.nq):
            px, py, phi, vx, vy, om = (A[:, self.ix(i, s)] for s in range(6))
            u1, u2 = A[:, self.iu(i, 0)], A[:, self.iu(i, 1)]
            S = u1 + u2
            sx = sum((A[:, self.ix(j, 0)] - px for j in self.neighbours(i)), np.zeros(A.shape[0]))
            sy = sum((A[:, self.ix(j, 1)] - py for j in self.neighbours(i)), np.zeros(A.shape[0]))
            out[:, self.ix(i, 0)] = px + dt * vx
            out[:, self.ix(i, 1)] = py + dt * vy
            out[:, self.ix(i, 2)] = phi + dt * om
            out[:, self.ix(i, 3)] = vx + dt * (-(S / m) * np.sin(phi) + (self.k / m) * sx)
            out[:, self.ix(i, 4)] = vy + dt * ((S / m) * np.cos(phi) - self.g + (self.k / m) * sy)
            out[:, self.ix(i, 5)] = om + dt * (self.arm / self.I) * (u2 - u1)
        return out

    def jacobian(self, alpha: np.ndarray) -> np.ndarray:
        """[A_k  B_k] = d f / d[x; u] at alpha (Eq. 8), dense [n_x, n]."""
        a = np.asarray(alpha, np.float64)
        J = np.zeros((self.n_x, self.n))
        dt, m = self.dt, self.m
        for i in range(self.nq):
            phi = a[self.ix(i, 2)]
            S = a[self.iu(i, 0)] + a[self.iu(i, 1)]
            for s in range(6):
                J[self.ix(i, s), self.ix(i, s)] = 1.0
            J[self.ix(i, 0), self.ix(i, 3)] = dt
            J[self.ix(i, 1), self.ix(i, 4)] = dt
            J[self.ix(i, 2), self.ix(i, 5)] = dt
            # v_x row
            J[self.ix(i, 3), self.ix(i, 2)] = -(dt / m) * S * math.cos(phi)
            J[self.ix(i, 3), self.iu(i, 0)] = -(dt / m) * math.sin(phi)
            J[self.ix(i, 3), self.iu(i, 1)] = -(dt / m) * math.sin(phi)
            # v_y row
            J[self.ix(i, 4), self.ix(i, 2)] = -(dt / m) * S * math.sin(phi)
            J[self.ix(i, 4), self.iu(i, 0)] = (dt / m) * math.cos(phi)
            J[self.ix(i, 4), self.iu(i, 1)] = (dt / m) * math.cos(phi)
            # omega row
            J[self.ix(i, 5), self.iu(i, 0)] = -dt * self.arm / self.I
            J[self.ix(i, 5), self.iu(i, 1)] = dt * self.arm / self.I
            # springs
            for j in self.neighbours(i):
                for s in (0, 1):
                    J[self.ix(i, 3 + s), self.ix(j, s)] += dt * self.k / m
                    J[self.ix(i, 3 + s), self.ix(i, s)] -= dt * self.k / m
        return J

    # Hessian entries ------------------------------------------------------------------------
    def hessian_terms(self, row: int):
        """Structurally nonzero entries H_{row, k j} = d^2 f_row / d alpha_k d alpha_j with j <= k.

        Returns a list of (j, k, fn) where fn(lo, hi) encloses the entry over the box [lo, hi]
        (the interval extension of the hand-derived second derivative). Springs are linear, so only
        the v_x and v_y rows are curved, through (phi, u_1, u_2) of their own quadrotor:

            v_x row:  H_{phi phi} = (dt/m) S sin(phi),   H_{u_r phi} = -(dt/m) cos(phi)
            v_y row:  H_{phi phi} = -(dt/m) S cos(phi),  H_{u_r phi} = -(dt/m) sin(phi)
        """
        i, s = divmod(row, 6)
        if s not in (3, 4):
            return []
        c = self.dt / self.m
        jp, j1, j2 = self.ix(i, 2), self.iu(i, 0), self.iu(i, 1)

        def S_iv(lo, hi):
            return (lo[j1] + lo[j2], hi[j1] + hi[j2])

        if s == 3:
            def h_pp(lo, hi):
                return iv_scale(c, iv_mul(S_iv(lo, hi), iv_sin(lo[jp], hi[jp])))

            def h_up(lo, hi):
                return iv_scale(-c, iv_cos(lo[jp], hi[jp]))
        else:
            def h_pp(lo, hi):
                return iv_scale(-c, iv_mul(S_iv(lo, hi), iv_cos(lo[jp], hi[jp])))

            def h_up(lo, hi):
                return iv_scale(-c, iv_sin(lo[jp], hi[jp]))
        return [(jp, jp, h_pp), (jp, j1, h_up), (jp, j2, h_up)]

    def hessian_point(self, alpha: np.ndarray) -> np.ndarray:
        """Dense Hessian tensor [n_x, n, n] at a point (from the same entry table)."""
        H = np.zeros((self.n_x, self.n, self.n))
        a = np.asarray(alpha, np.float64)
        for row in range(self.n_x):
            for j, k, fn in self.hessian_terms(row):
                v = fn(a, a)[0]
                H[row, k, j] = v
                H[row, j, k] = v
        return H


# ---------------------------------------------------------------------------------------------
# plain FP64 interval helpers (round-to-nearest; intervals are (lo, hi) tuples)
# ---------------------------------------------------------------------------------------------
def iv_add(a, b):
    return (a[0] + b[0], a[1] + b[1])


def iv_mul(a, b):
    p = (a[0] * b[0], a[0] * b[1], a[1] * b[0], a[1] * b[1])
    return (min(p), max(p))


def iv_scale(c: float, a):
    return (c * a[0], c * a[1]) if c >= 0 else (c * a[1], c * a[0])


def iv_sqr(a):
    """{d^2 : d in a} — the interval of squares (keeps non-negativity, Eq. 13)."""
    lo, hi = a
    if lo >= 0:
        return (lo * lo, hi * hi)
    if hi <= 0:
        return (hi * hi, lo * lo)
    return (0.0, max(lo * lo, hi * hi))


def _contains_point(lo: float, hi: float, offset: float, period: float) -> bool:
    """Is there an integer q with offset + q*period in [lo, hi]?"""
    q = math.ceil((lo - offset) / period)
    return offset + q * period <= hi


def iv_sin(lo: float, hi: float):
    """Exact range of sin over [lo, hi]: endpoints plus the extrema pi/2 + 2 pi q, -pi/2 + 2 pi q."""
    if hi - lo >= 2 * math.pi:
        return (-1.0, 1.0)
    vals = [math.sin(lo), math.sin(hi)]
    top = 1.0 if _contains_point(lo, hi, math.pi / 2, 2 * math.pi) else max(vals)
    bot = -1.0 if _contains_point(lo, hi, -math.pi / 2, 2 * math.pi) else min(vals)
    return (bot, top)


def iv_cos(lo: float, hi: float):
    """Exact range of cos over [lo, hi]: endpoints plus the extrema 2 pi q, pi + 2 pi q."""
    if hi - lo >= 2 * math.pi:
        return (-1.0, 1.0)
    vals = [math.cos(lo), math.cos(hi)]
    top = 1.0 if _contains_point(lo, hi, 0.0, 2 * math.pi) else max(vals)
    bot = -1.0 if _contains_point(lo, hi, math.pi, 2 * math.pi) else min(vals)
    return (bot, top)
