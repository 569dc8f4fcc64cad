"""Gradient of the path-based Hessian bound (Thm. 1) for differentiable LEBs (Sec. IV-D), plain FP64.

Test infrastructure (the oracle), not part of the product path.

The paper calls for LEBs that are differentiable in the nominal point (Sec. IV-D) and optimises nominal
points by projected gradient descent on the PBH bound's width (Sec. VI-A, Table II). The bound is a
piecewise-smooth function of the nominal point and the tube radii: interval endpoints are minima and
maxima of endpoint values, and the range of sin / cos over an interval is either an endpoint value or an
interior extremum (+-1). Its gradient here is that of the same algorithm with every such selection
fixed at the evaluation point, i.e. what automatic differentiation of Thm. 1 gives; where two candidates
of a minimum or maximum are exactly equal (a kink) it is the average of their derivatives (torch's
convention for min / max). It is obtained by
evaluating Thm. 1 once more with FP64 torch tensors (the same steps as ``oracle.pbh.pbh``: box set
centred at the nominal, displacement set, prefix sets X^(j), one interval term per structurally nonzero
Hessian entry, Eq. 15) and back-propagating through it.

Pinned (tests/test_oracle_pbh_grad.py) against central finite differences of ``oracle.pbh.pbh`` (an
independent NumPy implementation of the bound), against ``oracle.pbh.pbh`` for the values, and against a
hand-derived closed form at phi~ = 0.
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64


# ---- interval helpers on (lo, hi) pairs of 0-d FP64 tensors ------------------------------------------
def _mul(a, b):
    p = torch.stack([a[0] * b[0], a[0] * b[1], a[1] * b[0], a[1] * b[1]])
    return (p.min(), p.max())


def _scale(c: float, a):
    return (c * a[0], c * a[1]) if c >= 0 else (c * a[1], c * a[0])


def _scale_t(c, a):
    """c a for a tensor scalar c (sign taken at the evaluation point)."""
    return (c * a[0], c * a[1]) if _f(c) >= 0 else (c * a[1], c * a[0])


def _add(a, b):
    return (a[0] + b[0], a[1] + b[1])


def _sqr(a):
    lo, hi = a
    if _f(lo) >= 0:
        return (lo * lo, hi * hi)
    if _f(hi) <= 0:
        return (hi * hi, lo * lo)
    return (torch.zeros((), dtype=DT), torch.maximum(lo * lo, hi * hi))


def _f(x) -> float:
    return float(x.detach()) if torch.is_tensor(x) else float(x)


def _contains(lo: float, hi: float, offset: float, period: float) -> bool:
    q = math.ceil((lo - offset) / period)
    return offset + q * period <= hi


def _sin(lo, hi):
    """Range of sin over [lo, hi]: an endpoint value, or +-1 where an extremum lies inside."""
    if _f(hi) - _f(lo) >= 2 * math.pi:
        return (torch.tensor(-1.0, dtype=DT), torch.tensor(1.0, dtype=DT))
    s0, s1 = torch.sin(lo), torch.sin(hi)
    top = torch.tensor(1.0, dtype=DT) if _contains(_f(lo), _f(hi), math.pi / 2, 2 * math.pi) else torch.maximum(s0, s1)
    bot = torch.tensor(-1.0, dtype=DT) if _contains(_f(lo), _f(hi), -math.pi / 2, 2 * math.pi) else torch.minimum(s0, s1)
    return (bot, top)


def _cos(lo, hi):
    if _f(hi) - _f(lo) >= 2 * math.pi:
        return (torch.tensor(-1.0, dtype=DT), torch.tensor(1.0, dtype=DT))
    c0, c1 = torch.cos(lo), torch.cos(hi)
    top = torch.tensor(1.0, dtype=DT) if _contains(_f(lo), _f(hi), 0.0, 2 * math.pi) else torch.maximum(c0, c1)
    bot = torch.tensor(-1.0, dtype=DT) if _contains(_f(lo), _f(hi), math.pi, 2 * math.pi) else torch.minimum(c0, c1)
    return (bot, top)


def pbh_torch(dyn, alpha: torch.Tensor, radii: torch.Tensor):
    """Thm. 1 bound of a quadrotor chain (``oracle.dynamics.QuadChain``) over the box set of the given
    radii centred at the nominal alpha (hulled with the nominal). Returns (R_lo, R_hi) [n_x] FP64 tensors
    that carry gradients to alpha and radii.

    Rows of quadrotor i that are curved (Hessian table of ``QuadChain.hessian_terms``), with c = dt/m,
    S = u_1 + u_2, all entries involving (phi, u_1, u_2) of that quadrotor:
        v_x: H_{phi phi} = c S sin(phi),  H_{u_r phi} = -c cos(phi)
        v_y: H_{phi phi} = -c S cos(phi), H_{u_r phi} = -c sin(phi)
    In the natural path order phi precedes u_1, u_2, so every entry is evaluated over X^(phi): phi ranges
    over the box, the inputs sit at the nominal."""
    n_x = dyn.n_x
    lo = torch.minimum(alpha - radii, alpha)
    hi = torch.maximum(alpha + radii, alpha)
    D = [(lo[i] - alpha[i], hi[i] - alpha[i]) for i in range(dyn.n)]
    c = dyn.dt / dyn.m
    R_lo = [torch.zeros((), dtype=DT) for _ in range(n_x)]
    R_hi = [torch.zeros((), dtype=DT) for _ in range(n_x)]
    for i in range(dyn.nq):
        jp, j1, j2 = dyn.ix(i, 2), dyn.iu(i, 0), dyn.iu(i, 1)
        # prefix set X^(phi): phi over [lo, hi]; u_1, u_2 later in the path order, at the nominal
        S = alpha[j1] + alpha[j2]
        sin_iv = _sin(lo[jp], hi[jp])
        cos_iv = _cos(lo[jp], hi[jp])
        for s, h_pp, h_up in ((3, _scale_t(c * S, sin_iv), _scale(-c, cos_iv)),
                              (4, _scale_t(-c * S, cos_iv), _scale(-c, sin_iv))):
            R = _scale(0.5, _mul(h_pp, _sqr(D[jp])))                 # 1/2 [H_pp] Delta_phi^2
            R = _add(R, _mul(h_up, _mul(D[jp], D[j1])))             # [H_u1 phi] Delta_phi Delta_u1
            R = _add(R, _mul(h_up, _mul(D[jp], D[j2])))             # [H_u2 phi] Delta_phi Delta_u2
            R_lo[dyn.ix(i, s)], R_hi[dyn.ix(i, s)] = R
    return torch.stack(R_lo), torch.stack(R_hi)


def pbh_vjp(dyn, nominal: np.ndarray, radii: np.ndarray, g_lo: np.ndarray, g_hi: np.ndarray):
    """d(g_lo . R_lo + g_hi . R_hi) / d(x~, u~, radii) of Thm. 1 at one timestep (box set centred at the
    nominal). Returns (g_x [n_x], g_u [n_u], g_radii [n]) FP64."""
    a = torch.tensor(np.asarray(nominal, np.float64), dtype=DT, requires_grad=True)
    r = torch.tensor(np.asarray(radii, np.float64), dtype=DT, requires_grad=True)
    R_lo, R_hi = pbh_torch(dyn, a, r)
    L = (torch.tensor(np.asarray(g_lo, np.float64)) * R_lo).sum() + (torch.tensor(np.asarray(g_hi, np.float64)) * R_hi).sum()
    ga, gr = torch.autograd.grad(L, (a, r), allow_unused=True)
    ga = torch.zeros_like(a) if ga is None else ga
    gr = torch.zeros_like(r) if gr is None else gr
    ga, gr = ga.numpy(), gr.numpy()
    return ga[: dyn.n_x], ga[dyn.n_x:], gr


def width(dyn, nominal: np.ndarray, radii: np.ndarray) -> float:
    """Summed width sum_l (R_hi - R_lo) of the Thm. 1 bound at one timestep (the objective of the
    nominal optimisation of Table II)."""
    a = torch.tensor(np.asarray(nominal, np.float64), dtype=DT)
    r = torch.tensor(np.asarray(radii, np.float64), dtype=DT)
    R_lo, R_hi = pbh_torch(dyn, a, r)
    return float((R_hi - R_lo).sum())
