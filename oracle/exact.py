"""Exact ranges of the linearization error (Eq. 9c / Eq. 10) on small problems, FP64.

These are independent of the bounding methods: a sound bound (Thm. 1 or Thm. 3) must contain them.

* ``quad_exact_range``: the planar quadrotor (and each quadrotor of the spring chain, whose springs are
  linear) has curved rows v_x and v_y only. With S = u_1 + u_2, dS = du_1 + du_2 and phi = phi~ + dphi,
  the remainder w.r.t. the exact Jacobian is

      r_vx = -(dt/m) [ S~ (sin phi - sin phi~ - cos phi~ dphi) + dS (sin phi - sin phi~) ]
      r_vy =  (dt/m) [ S~ (cos phi - cos phi~ + sin phi~ dphi) + dS (cos phi - cos phi~) ]

  Both are affine in dS (extremes at its endpoints) and, for fixed dS, smooth in phi with stationary
  points where (S~ + dS) cos phi = S~ cos phi~ (v_x) or (S~ + dS) sin phi = S~ sin phi~ (v_y). The
  exact range is the min/max over those finitely many candidates. All other rows are exactly zero.

* ``relu_exact_range``: a ReLU network is piecewise affine. Activation patterns of the neurons that are
  unstable over the box are enumerated depth-first; a branch is kept only if its polytope is non-empty
  (linear program). On each leaf the remainder r(alpha) = f(alpha) - f(alpha~) - J (alpha - alpha~) is
  affine, so its min and max over the leaf polytope are two linear programs per output row.
"""
from __future__ import annotations

import math
import numpy as np
from scipy.optimize import linprog


# ------------------------------------------------------------------------------------------------
def _angles_with_cos(c: float, lo: float, hi: float):
    if not -1.0 <= c <= 1.0:
        return []
    base = math.acos(c)
    out = []
    for b in (base, -base):
        q0 = math.ceil((lo - b) / (2 * math.pi))
        q = q0
        while b + 2 * math.pi * q <= hi:
            out.append(b + 2 * math.pi * q)
            q += 1
    return out


def _angles_with_sin(s: float, lo: float, hi: float):
    if not -1.0 <= s <= 1.0:
        return []
    base = math.asin(s)
    out = []
    for b in (base, math.pi - base):
        q0 = math.ceil((lo - b) / (2 * math.pi))
        q = q0
        while b + 2 * math.pi * q <= hi:
            out.append(b + 2 * math.pi * q)
            q += 1
    return out


def quad_exact_range(dyn, nominal: np.ndarray, lo: np.ndarray, hi: np.ndarray):
    """Exact [min, max] of each row's remainder over the box, for a QuadChain model."""
    a = np.asarray(nominal, np.float64)
    r_lo = np.zeros(dyn.n_x)
    r_hi = np.zeros(dyn.n_x)
    c = dyn.dt / dyn.m
    for i in range(dyn.nq):
        jp, j1, j2 = dyn.ix(i, 2), dyn.iu(i, 0), dyn.iu(i, 1)
        ph0 = a[jp]
        S0 = a[j1] + a[j2]
        dS_ends = (lo[j1] - a[j1] + lo[j2] - a[j2], hi[j1] - a[j1] + hi[j2] - a[j2])
        plo, phi_hi = lo[jp], hi[jp]

        def rvx(ph, dS):
            return -c * (S0 * (math.sin(ph) - math.sin(ph0) - math.cos(ph0) * (ph - ph0))
                         + dS * (math.sin(ph) - math.sin(ph0)))

        def rvy(ph, dS):
            return c * (S0 * (math.cos(ph) - math.cos(ph0) + math.sin(ph0) * (ph - ph0))
                        + dS * (math.cos(ph) - math.cos(ph0)))

        vx_vals, vy_vals = [], []
        for dS in dS_ends:
            S = S0 + dS
            cand_x = [plo, phi_hi]
            cand_y = [plo, phi_hi]
            if S != 0.0:
                cand_x += _angles_with_cos(S0 * math.cos(ph0) / S, plo, phi_hi)
                cand_y += _angles_with_sin(S0 * math.sin(ph0) / S, plo, phi_hi)
            vx_vals += [rvx(p, dS) for p in cand_x]
            vy_vals += [rvy(p, dS) for p in cand_y]
        r_lo[dyn.ix(i, 3)], r_hi[dyn.ix(i, 3)] = min(vx_vals), max(vx_vals)
        r_lo[dyn.ix(i, 4)], r_hi[dyn.ix(i, 4)] = min(vy_vals), max(vy_vals)
    return r_lo, r_hi


# ------------------------------------------------------------------------------------------------
def _lp_extreme(cvec, A_ub, b_ub, bounds, maximize: bool):
    res = linprog(-cvec if maximize else cvec, A_ub=A_ub if len(A_ub) else None,
                  b_ub=b_ub if len(b_ub) else None, bounds=bounds, method="highs")
    if res.status != 0:
        return None
    return -res.fun if maximize else res.fun


def relu_exact_range(Ws, bs, nominal, lo, hi, lin=None, residual=True, cap: int = 10000):
    """Exact [min, max] of r(alpha) = f(alpha) - f(alpha~) - lin (alpha - alpha~) over the box.

    ``lin`` defaults to the exact Jacobian of f at the nominal (all nominal pre-activations nonzero).
    Returns (r_lo, r_hi, n_regions)."""
    Ws = [np.asarray(W, np.float64) for W in Ws]
    bs = [np.asarray(b, np.float64) for b in bs]
    a = np.asarray(nominal, np.float64)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    n = a.shape[0]
    n_x = Ws[-1].shape[0]

    # nominal value and Jacobian
    h = a
    Jm = np.eye(n)
    for W, b in zip(Ws[:-1], bs[:-1]):
        z = W @ h + b
        D = (z > 0).astype(np.float64)
        Jm = D[:, None] * (W @ Jm)
        h = np.maximum(z, 0.0)
    f_nom = Ws[-1] @ h + bs[-1]
    J = Ws[-1] @ Jm
    if residual:
        f_nom = f_nom + a[:n_x]
        J = J.copy()
        J[:, :n_x] += np.eye(n_x)
    if lin is None:
        lin = J
    lin = np.asarray(lin, np.float64)
    bnds = list(zip(lo, hi))

    r_lo = np.full(n_x, np.inf)
    r_hi = np.full(n_x, -np.inf)
    count = [0]

    def leaf(P, q, A_ub, b_ub):
        # output affine map on this region: f(alpha) = P alpha + q
        count[0] += 1
        if count[0] > cap:
            raise RuntimeError("region cap exceeded")
        Pf = P.copy()
        qf = q.copy()
        if residual:
            Pf[:, :n_x] += np.eye(n_x)
        C = Pf - lin                              # r(alpha) = C alpha + d
        d = qf - f_nom + lin @ a
        for row in range(n_x):
            mn = _lp_extreme(C[row], A_ub, b_ub, bnds, False)
            mx = _lp_extreme(C[row], A_ub, b_ub, bnds, True)
            r_lo[row] = min(r_lo[row], mn + d[row])
            r_hi[row] = max(r_hi[row], mx + d[row])

    def descend(layer, P, q, A_ub, b_ub):
        # P, q: affine map alpha -> input of this layer (h_{layer}) on the current region
        W, b = Ws[layer], bs[layer]
        Pz = W @ P
        qz = W @ q + b
        if layer == len(Ws) - 1:
            leaf(Pz, qz, A_ub, b_ub)
            return
        m = W.shape[0]
        state = np.zeros(m)          # +1 active, -1 inactive, 0 undecided
        for j in range(m):
            mn = _lp_extreme(Pz[j], A_ub, b_ub, bnds, False)
            mx = _lp_extreme(Pz[j], A_ub, b_ub, bnds, True)
            if mn is None:
                return
            if mn + qz[j] >= 0:
                state[j] = 1
            elif mx + qz[j] <= 0:
                state[j] = -1
        undecided = [j for j in range(m) if state[j] == 0]

        def branch(idx, st, A, bvec):
            if idx == len(undecided):
                D = (st > 0).astype(np.float64)
                descend(layer + 1, D[:, None] * Pz, D * qz, A, bvec)
                return
            j = undecided[idx]
            for sign in (1, -1):
                # active: z_j >= 0  <=>  -Pz_j alpha <= qz_j ; inactive: Pz_j alpha <= -qz_j
                row = -Pz[j] if sign > 0 else Pz[j]
                rhs = qz[j] if sign > 0 else -qz[j]
                A2 = np.vstack([A, row[None, :]]) if len(A) else row[None, :]
                b2 = np.append(bvec, rhs)
                if _lp_extreme(np.zeros(n), A2, b2, bnds, False) is None:
                    continue
                st2 = st.copy()
                st2[j] = sign
                branch(idx + 1, st2, A2, b2)

        branch(0, state, A_ub, b_ub)

    descend(0, np.eye(n), np.zeros(n), np.zeros((0, n)), np.zeros(0))
    return r_lo, r_hi, count[0]
