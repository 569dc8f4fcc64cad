"""The paper's satellite and (coupled) 3-D quadrotor dynamics (App. A) in FP64: model, Jacobian (Eq. 8)
and the hand-derived Hessian entries with their interval extensions for Thm. 1.

Test infrastructure (the oracle), not part of the product path.

Both are integrated by forward Euler, x+ = x + dt xdot(x, u). The model and its Jacobian / Hessian at a
point are evaluated with FP64 torch tensors (automatic differentiation, a library step), which pins the
hand-derived Hessian table used by Thm. 1 (``hessian_terms``; tests/test_oracle_dynamics3d.py).

Satellite (App. A "Satellite"): state (q_0..q_3, w_1..w_3), input torque (v_1..v_3),
    qdot = 1/2 zeta(w) q,  wdot = I_S^-1 (v - w x (I_S w)),  I_S = diag(I_1, I_2, I_3),
the "w" of the paper's cross product read as the rotation rate w. Every entry is bilinear, so the
Hessian is constant:
    q_0: d2/dw_a dq_a = -dt/2 (a = 1..3)
    q_1: (w_1, q_0) +dt/2, (w_3, q_2) +dt/2, (w_2, q_3) -dt/2
    q_2: (w_2, q_0) +dt/2, (w_3, q_1) -dt/2, (w_1, q_3) +dt/2
    q_3: (w_3, q_0) +dt/2, (w_2, q_1) +dt/2, (w_1, q_2) -dt/2
    w_1: (w_2, w_3) dt (I_2 - I_3)/I_1;  w_2: (w_1, w_3) dt (I_3 - I_1)/I_2;  w_3: (w_1, w_2) dt (I_1 - I_2)/I_3

3-D quadrotor (App. A "Coupled 3D Quadrotor"), per quadrotor
    state (p_x, p_y, p_z, phi, theta, psi, v_x, v_y, v_z, p, q, r), input (T, tau_phi, tau_theta, tau_psi),
states of all quadrotors first, then inputs; the centroid spring-damper of the coupled system adds
-alpha N (p_i - pbar) - gamma (v_i - vbar) to the translational accelerations (linear: no Hessian term).
With a = q sin(phi) + r cos(phi) the curved rows and their second derivatives (j <= k in path order
phi < theta < psi < p < q < r < T):
    phidot   = p + a tan(theta)
    thetadot = q cos(phi) - r sin(phi)
    psidot   = a / cos(theta)
    v_x dot  = (T/m) g_x, g_x = cos(psi) sin(theta) cos(phi) + sin(psi) sin(phi)
    v_y dot  = (T/m) g_y, g_y = sin(psi) sin(theta) cos(phi) - cos(psi) sin(phi)
    v_z dot  = (T/m) cos(theta) cos(phi) - g
    pdot = (J_y - J_z)/J_x q r + tau_phi/J_x, qdot = (J_z - J_x)/J_y p r + ..., rdot = (J_x - J_y)/J_z p q + ...
(entries listed in ``Quad3D._row_terms``). Every entry is evaluated over the prefix set X^(j) of its
smaller path index with the natural interval extension of the expression (interval sin/cos, tan and sec
over an interval inside (-pi/2, pi/2), interval products and sums).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .dynamics import iv_add, iv_cos, iv_mul, iv_scale, iv_sin

DT = torch.float64


def iv_neg(a):
    return (-a[1], -a[0])


def iv_pt(v: float):
    return (v, v)


def iv_tan(lo: float, hi: float):
    """Range of tan over [lo, hi] inside (-pi/2, pi/2) (increasing there)."""
    if not (-math.pi / 2 < lo and hi < math.pi / 2):
        return (-math.inf, math.inf)
    return (math.tan(lo), math.tan(hi))


def iv_sec(lo: float, hi: float):
    """Range of 1/cos over [lo, hi] inside (-pi/2, pi/2): cos > 0 there, 1/cos = sec."""
    if not (-math.pi / 2 < lo and hi < math.pi / 2):
        return (-math.inf, math.inf)
    c = iv_cos(lo, hi)
    return (1.0 / c[1], 1.0 / c[0])


def _jac_hess(fn, alpha: np.ndarray, n_x: int):
    a = torch.tensor(np.asarray(alpha, np.float64), dtype=DT)
    J = torch.autograd.functional.jacobian(fn, a)
    H = torch.stack([torch.autograd.functional.hessian(lambda z, l=l: fn(z)[l], a) for l in range(n_x)])
    return J.numpy(), H.numpy()


class Satellite:
    def __init__(self, dt: float = 0.05, inertia=(5.0, 2.0, 1.0), **_):
        self.dt = float(dt)
        self.I = tuple(float(v) for v in inertia)
        self.n_x, self.n_u = 7, 3
        self.n = 10

    def xdot_t(self, a: torch.Tensor) -> torch.Tensor:
        q0, q1, q2, q3, w1, w2, w3, v1, v2, v3 = (a[..., i] for i in range(10))
        I1, I2, I3 = self.I
        qd = torch.stack([0.5 * (-w1 * q1 - w2 * q2 - w3 * q3),
                          0.5 * (w1 * q0 + w3 * q2 - w2 * q3),
                          0.5 * (w2 * q0 - w3 * q1 + w1 * q3),
                          0.5 * (w3 * q0 + w2 * q1 - w1 * q2)], -1)
        # w x (I w) = ((I3 - I2) w2 w3, (I1 - I3) w1 w3, (I2 - I1) w1 w2)
        wd = torch.stack([(v1 - (I3 - I2) * w2 * w3) / I1,
                          (v2 - (I1 - I3) * w1 * w3) / I2,
                          (v3 - (I2 - I1) * w1 * w2) / I3], -1)
        return torch.cat([qd, wd], -1)

    def f_t(self, a: torch.Tensor) -> torch.Tensor:
        return a[..., :7] + self.dt * self.xdot_t(a)

    def f(self, alpha):
        return self.f_t(torch.tensor(np.asarray(alpha, np.float64), dtype=DT)).numpy()

    def f_batch(self, A):
        return self.f_t(torch.tensor(np.asarray(A, np.float64), dtype=DT)).numpy()

    def jacobian(self, alpha):
        a = torch.tensor(np.asarray(alpha, np.float64), dtype=DT)
        return torch.autograd.functional.jacobian(self.f_t, a).numpy()

    def hessian_autodiff(self, alpha):
        return _jac_hess(self.f_t, alpha, self.n_x)[1]

    def _entries(self):
        h = 0.5 * self.dt
        I1, I2, I3 = self.I
        # (row, j, k, value) with j < k in the natural order (q before w)
        return [(0, 1, 4, -h), (0, 2, 5, -h), (0, 3, 6, -h),
                (1, 0, 4, h), (1, 2, 6, h), (1, 3, 5, -h),
                (2, 0, 5, h), (2, 1, 6, -h), (2, 3, 4, h),
                (3, 0, 6, h), (3, 1, 5, h), (3, 2, 4, -h),
                (4, 5, 6, self.dt * (I2 - I3) / I1), (5, 4, 6, self.dt * (I3 - I1) / I2),
                (6, 4, 5, self.dt * (I1 - I2) / I3)]

    def hessian_terms(self, row: int):
        return [(j, k, (lambda lo, hi, v=v: (v, v))) for r, j, k, v in self._entries() if r == row]

    def hessian_point(self, alpha):
        H = np.zeros((self.n_x, self.n, self.n))
        for r, j, k, v in self._entries():
            H[r, j, k] = H[r, k, j] = v
        return H


class Quad3D:
    """n_quads 3-D quadrotors, optionally coupled by the centroid spring-damper (alpha, gamma)."""

    def __init__(self, n_quads: int = 1, dt: float = 0.05, mass: float = 1.0, g: float = 9.81,
                 inertia=(0.01, 0.01, 0.02), coup_alpha: float = 0.0, coup_gamma: float = 0.0, **_):
        self.nq = int(n_quads)
        self.dt, self.m, self.g = float(dt), float(mass), float(g)
        self.J = tuple(float(v) for v in inertia)
        self.alpha, self.gamma = float(coup_alpha), float(coup_gamma)
        self.n_x, self.n_u = 12 * self.nq, 4 * self.nq
        self.n = self.n_x + self.n_u

    def ix(self, i: int, s: int) -> int:
        return 12 * i + s

    def iu(self, i: int, r: int) -> int:
        return self.n_x + 4 * i + r

    # ---- model ---------------------------------------------------------------------------------
    def xdot_t(self, a: torch.Tensor) -> torch.Tensor:
        N = self.nq
        X = a[..., : self.n_x].reshape(*a.shape[:-1], N, 12)
        U = a[..., self.n_x:].reshape(*a.shape[:-1], N, 4)
        px, py, pz, ph, th, ps, vx, vy, vz, p, q, r = (X[..., s] for s in range(12))
        T, tp, tt, tq = (U[..., s] for s in range(4))
        Jx, Jy, Jz = self.J
        sph, cph, sth, cth, sps, cps = (torch.sin(ph), torch.cos(ph), torch.sin(th), torch.cos(th), torch.sin(ps),
                                        torch.cos(ps))
        aa = q * sph + r * cph
        acc = [(T / self.m) * (cps * sth * cph + sps * sph), (T / self.m) * (sps * sth * cph - cps * sph),
               (T / self.m) * (cth * cph) - self.g]
        pos, vel = (px, py, pz), (vx, vy, vz)
        if self.alpha != 0.0 or self.gamma != 0.0:
            acc = [acc[d] - self.alpha * N * (pos[d] - pos[d].mean(-1, keepdim=True))
                   - self.gamma * (vel[d] - vel[d].mean(-1, keepdim=True)) for d in range(3)]
        out = torch.stack([vx, vy, vz, p + aa * torch.tan(th), q * cph - r * sph, aa / cth, acc[0], acc[1], acc[2],
                           (Jy - Jz) / Jx * q * r + tp / Jx, (Jz - Jx) / Jy * p * r + tt / Jy,
                           (Jx - Jy) / Jz * p * q + tq / Jz], -1)
        return out.reshape(*a.shape[:-1], self.n_x)

    def f_t(self, a: torch.Tensor) -> torch.Tensor:
        return a[..., : self.n_x] + self.dt * self.xdot_t(a)

    def f(self, alpha):
        return self.f_t(torch.tensor(np.asarray(alpha, np.float64), dtype=DT)).numpy()

    def f_batch(self, A):
        return self.f_t(torch.tensor(np.asarray(A, np.float64), dtype=DT)).numpy()

    def jacobian(self, alpha):
        a = torch.tensor(np.asarray(alpha, np.float64), dtype=DT)
        return torch.autograd.functional.jacobian(self.f_t, a).numpy()

    def hessian_autodiff(self, alpha):
        return _jac_hess(self.f_t, alpha, self.n_x)[1]

    # ---- Hessian table -----------------------------------------------------------------------
    def _row_terms(self, i: int, s: int):
        """Second derivatives of row s of quadrotor i (times dt), as (j, k, fn(lo, hi)) with j <= k;
        fn is the natural interval extension of the entry over the box [lo, hi]."""
        dt, m = self.dt, self.m
        jph, jth, jps = self.ix(i, 3), self.ix(i, 4), self.ix(i, 5)
        jp, jq, jr, jT = self.ix(i, 9), self.ix(i, 10), self.ix(i, 11), self.iu(i, 0)

        def V(lo, hi, j):
            return (lo[j], hi[j])

        def trig(lo, hi):
            return (iv_sin(lo[jph], hi[jph]), iv_cos(lo[jph], hi[jph]), iv_sin(lo[jth], hi[jth]),
                    iv_cos(lo[jth], hi[jth]), iv_sin(lo[jps], hi[jps]), iv_cos(lo[jps], hi[jps]))

        def A(lo, hi):      # a = q sin(phi) + r cos(phi)
            sph, cph = iv_sin(lo[jph], hi[jph]), iv_cos(lo[jph], hi[jph])
            return iv_add(iv_mul(V(lo, hi, jq), sph), iv_mul(V(lo, hi, jr), cph))

        def Aphi(lo, hi):   # a_phi = q cos(phi) - r sin(phi)
            sph, cph = iv_sin(lo[jph], hi[jph]), iv_cos(lo[jph], hi[jph])
            return iv_add(iv_mul(V(lo, hi, jq), cph), iv_neg(iv_mul(V(lo, hi, jr), sph)))

        def tanT(lo, hi):
            return iv_tan(lo[jth], hi[jth])

        def secT(lo, hi):
            return iv_sec(lo[jth], hi[jth])

        def sq(x):
            return iv_mul(x, x) if x[0] >= 0 or x[1] <= 0 else (0.0, max(x[0] * x[0], x[1] * x[1]))

        S = lambda c, x: iv_scale(c, x)
        if s == 3:   # phidot = p + a tan(theta)
            return [
                (jph, jph, lambda lo, hi: S(-dt, iv_mul(A(lo, hi), tanT(lo, hi)))),
                (jph, jth, lambda lo, hi: S(dt, iv_mul(Aphi(lo, hi), sq(secT(lo, hi))))),
                (jth, jth, lambda lo, hi: S(2 * dt, iv_mul(A(lo, hi), iv_mul(sq(secT(lo, hi)), tanT(lo, hi))))),
                (jph, jq, lambda lo, hi: S(dt, iv_mul(iv_cos(lo[jph], hi[jph]), tanT(lo, hi)))),
                (jph, jr, lambda lo, hi: S(-dt, iv_mul(iv_sin(lo[jph], hi[jph]), tanT(lo, hi)))),
                (jth, jq, lambda lo, hi: S(dt, iv_mul(iv_sin(lo[jph], hi[jph]), sq(secT(lo, hi))))),
                (jth, jr, lambda lo, hi: S(dt, iv_mul(iv_cos(lo[jph], hi[jph]), sq(secT(lo, hi))))),
            ]
        if s == 4:   # thetadot = q cos(phi) - r sin(phi)
            return [
                (jph, jph, lambda lo, hi: S(-dt, Aphi(lo, hi))),
                (jph, jq, lambda lo, hi: S(-dt, iv_sin(lo[jph], hi[jph]))),
                (jph, jr, lambda lo, hi: S(-dt, iv_cos(lo[jph], hi[jph]))),
            ]
        if s == 5:   # psidot = a sec(theta)
            return [
                (jph, jph, lambda lo, hi: S(-dt, iv_mul(A(lo, hi), secT(lo, hi)))),
                (jph, jth, lambda lo, hi: S(dt, iv_mul(Aphi(lo, hi), iv_mul(secT(lo, hi), tanT(lo, hi))))),
                (jth, jth, lambda lo, hi: S(dt, iv_mul(A(lo, hi), iv_mul(secT(lo, hi),
                                                                        iv_add(sq(tanT(lo, hi)), sq(secT(lo, hi))))))),
                (jph, jq, lambda lo, hi: S(dt, iv_mul(iv_cos(lo[jph], hi[jph]), secT(lo, hi)))),
                (jph, jr, lambda lo, hi: S(-dt, iv_mul(iv_sin(lo[jph], hi[jph]), secT(lo, hi)))),
                (jth, jq, lambda lo, hi: S(dt, iv_mul(iv_sin(lo[jph], hi[jph]), iv_mul(secT(lo, hi), tanT(lo, hi))))),
                (jth, jr, lambda lo, hi: S(dt, iv_mul(iv_cos(lo[jph], hi[jph]), iv_mul(secT(lo, hi), tanT(lo, hi))))),
            ]
        if s in (6, 7):
            # g and its partials as interval expressions in (phi, theta, psi); T/m and 1/m factors
            def g_parts(lo, hi):
                sph, cph, sth, cth, sps, cps = trig(lo, hi)
                m_ = iv_mul
                if s == 6:   # g_x = c_psi s_th c_ph + s_psi s_ph
                    g = iv_add(m_(m_(cps, sth), cph), m_(sps, sph))
                    g_ph = iv_add(iv_neg(m_(m_(cps, sth), sph)), m_(sps, cph))
                    g_th = m_(m_(cps, cth), cph)
                    g_ps = iv_add(iv_neg(m_(m_(sps, sth), cph)), m_(cps, sph))
                    g_phth = iv_neg(m_(m_(cps, cth), sph))
                    g_phps = iv_add(m_(m_(sps, sth), sph), m_(cps, cph))
                    g_thth = iv_neg(m_(m_(cps, sth), cph))
                    g_thps = iv_neg(m_(m_(sps, cth), cph))
                else:        # g_y = s_psi s_th c_ph - c_psi s_ph
                    g = iv_add(m_(m_(sps, sth), cph), iv_neg(m_(cps, sph)))
                    g_ph = iv_add(iv_neg(m_(m_(sps, sth), sph)), iv_neg(m_(cps, cph)))
                    g_th = m_(m_(sps, cth), cph)
                    g_ps = iv_add(m_(m_(cps, sth), cph), m_(sps, sph))
                    g_phth = iv_neg(m_(m_(sps, cth), sph))
                    g_phps = iv_add(iv_neg(m_(m_(cps, sth), sph)), m_(sps, cph))
                    g_thth = iv_neg(m_(m_(sps, sth), cph))
                    g_thps = m_(m_(cps, cth), cph)
                return dict(g=g, ph=g_ph, th=g_th, ps=g_ps, phph=iv_neg(g), phth=g_phth, phps=g_phps, thth=g_thth,
                            thps=g_thps, psps=iv_neg(g))

            def Tm(lo, hi):
                return iv_scale(dt / m, V(lo, hi, jT))

            return [
                (jph, jph, lambda lo, hi: iv_mul(Tm(lo, hi), g_parts(lo, hi)["phph"])),
                (jph, jth, lambda lo, hi: iv_mul(Tm(lo, hi), g_parts(lo, hi)["phth"])),
                (jph, jps, lambda lo, hi: iv_mul(Tm(lo, hi), g_parts(lo, hi)["phps"])),
                (jth, jth, lambda lo, hi: iv_mul(Tm(lo, hi), g_parts(lo, hi)["thth"])),
                (jth, jps, lambda lo, hi: iv_mul(Tm(lo, hi), g_parts(lo, hi)["thps"])),
                (jps, jps, lambda lo, hi: iv_mul(Tm(lo, hi), g_parts(lo, hi)["psps"])),
                (jph, jT, lambda lo, hi: S(dt / m, g_parts(lo, hi)["ph"])),
                (jth, jT, lambda lo, hi: S(dt / m, g_parts(lo, hi)["th"])),
                (jps, jT, lambda lo, hi: S(dt / m, g_parts(lo, hi)["ps"])),
            ]
        if s == 8:   # v_z dot = (T/m) cos(theta) cos(phi) - g
            def parts(lo, hi):
                sph, cph, sth, cth = (iv_sin(lo[jph], hi[jph]), iv_cos(lo[jph], hi[jph]), iv_sin(lo[jth], hi[jth]),
                                      iv_cos(lo[jth], hi[jth]))
                return dict(g=iv_mul(cth, cph), ph=iv_neg(iv_mul(cth, sph)), th=iv_neg(iv_mul(sth, cph)),
                            phth=iv_mul(sth, sph))

            def Tm(lo, hi):
                return iv_scale(dt / m, V(lo, hi, jT))

            return [
                (jph, jph, lambda lo, hi: iv_mul(Tm(lo, hi), iv_neg(parts(lo, hi)["g"]))),
                (jph, jth, lambda lo, hi: iv_mul(Tm(lo, hi), parts(lo, hi)["phth"])),
                (jth, jth, lambda lo, hi: iv_mul(Tm(lo, hi), iv_neg(parts(lo, hi)["g"]))),
                (jph, jT, lambda lo, hi: S(dt / m, parts(lo, hi)["ph"])),
                (jth, jT, lambda lo, hi: S(dt / m, parts(lo, hi)["th"])),
            ]
        Jx, Jy, Jz = self.J
        if s == 9:
            c = dt * (Jy - Jz) / Jx
            return [(jq, jr, lambda lo, hi, c=c: (c, c))]
        if s == 10:
            c = dt * (Jz - Jx) / Jy
            return [(jp, jr, lambda lo, hi, c=c: (c, c))]
        if s == 11:
            c = dt * (Jx - Jy) / Jz
            return [(jp, jq, lambda lo, hi, c=c: (c, c))]
        return []

    def hessian_terms(self, row: int):
        i, s = divmod(row, 12)
        return self._row_terms(i, s)

    def hessian_point(self, alpha):
        a = np.asarray(alpha, np.float64)
        H = np.zeros((self.n_x, self.n, self.n))
        for row in range(self.n_x):
            for j, k, fn in self.hessian_terms(row):
                v = fn(a, a)[0]
                H[row, j, k] = H[row, k, j] = v
        return H
