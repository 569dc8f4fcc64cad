"""CROWN affine bounds (Thm. 2) and the Jacobian-corrected remainder bound (Thm. 3), torch FP64 on CPU.

The network is f(alpha) = W_L h_{L-1} + b_L with h_i = sigma(W_i h_{i-1} + b_i), h_0 = alpha. With
``residual`` the dynamics are x+ = x + f([x; u]); the identity part is affine, so its CROWN bounds are
exact and it cancels in Thm. 3's remainder.

Thm. 2 (Zhang et al. 2018, Thm. 3.2) gives only the statement; its internals follow the cited work, with
these readings fixed so that the result is a single deterministic function:

* Layer-1 pre-activation bounds are exact: W_1 c +- |W_1| r + b_1 over the box (c, r).
* Every later layer's pre-activation bounds (and the output) come from full back-substitution to the
  input: start from the layer's rows Lambda = W_i, and for each earlier hidden layer pick, per neuron,
  the lower relaxation line where the coefficient is >= 0 and the upper line where it is < 0 (reversed
  for upper bounds), then move through that layer's affine map.
* ReLU lines: upper = chord u(z - l)/(u - l); lower slope 1 if u >= -l else 0 (stable neurons exact).
* tanh lines: l >= 0 -> upper tangent at (l+u)/2, lower chord; u <= 0 mirrored; l < 0 < u -> the tangent
  lines through the endpoints (tangent point by bisection), falling back to the chord when the tangent
  point leaves [l, u].
* Every intercept is the exact extremum of sigma(z) - s z over [l, u] (endpoints plus critical points),
  so each line is valid for whatever slope was chosen.

Thm. 3: r_lo = min_X (W_lo - J) alpha + J alpha~ - f(alpha~) + b_lo and r_hi = max_X (W_hi - J) alpha
+ J alpha~ - f(alpha~) + b_hi, each an affine function minimised/maximised over the box in closed form.

Everything is written with torch ops so that the bound is differentiable in (x~, u~, radii); the
tangent-point bisection is made differentiable by one implicit-function (Newton) step.
"""
from __future__ import annotations

import math
import torch

F64 = torch.float64


def act_fn(act: str, z: torch.Tensor) -> torch.Tensor:
    return torch.relu(z) if act == "relu" else torch.tanh(z)


def act_deriv(act: str, z: torch.Tensor) -> torch.Tensor:
    if act == "relu":
        return (z > 0).to(z.dtype)            # derivative 0 at the kink z = 0
    t = torch.tanh(z)
    return 1.0 - t * t


def forward(Ws, bs, act: str, alpha: torch.Tensor):
    """Returns (output, [pre-activations of the hidden layers])."""
    h = alpha
    zs = []
    for i, (W, b) in enumerate(zip(Ws, bs)):
        z = W @ h + b
        if i + 1 < len(Ws):
            zs.append(z)
            h = act_fn(act, z)
        else:
            return z, zs


def jacobian(Ws, bs, act: str, alpha: torch.Tensor) -> torch.Tensor:
    """J = W_L D_{L-1} W_{L-1} ... D_1 W_1 with D_i = diag(sigma'(z_i)) at alpha."""
    _, zs = forward(Ws, bs, act, alpha)
    J = Ws[0]
    for i in range(1, len(Ws)):
        J = Ws[i] @ (act_deriv(act, zs[i - 1])[:, None] * J)
    return J


# ------------------------------------------------------------------------------------------------
# relaxation lines
# ------------------------------------------------------------------------------------------------
def _tanh_tangent_from(l: torch.Tensor) -> torch.Tensor:
    """Tangent point d > 0 of the line through (l, tanh l), l < 0: tanh'(d)(d - l) = tanh d - tanh l."""
    def g(d, l_):
        return torch.tanh(d) - torch.tanh(l_) - (1 - torch.tanh(d) ** 2) * (d - l_)

    with torch.no_grad():
        lo = torch.zeros_like(l)
        hi = torch.full_like(l, 20.0)
        ld = l.detach()
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            pos = g(mid, ld) > 0
            hi = torch.where(pos, mid, hi)
            lo = torch.where(pos, lo, mid)
        d0 = 0.5 * (lo + hi)
    # one Newton step with d0 detached: same value, implicit-function derivative in l
    t = torch.tanh(d0)
    gd = -(-2 * t * (1 - t * t)) * (d0 - l)          # dg/dd = -tanh''(d)(d - l)
    return d0 - g(d0, l) / gd


def _critical_points(act: str, s: torch.Tensor):
    """Points where sigma'(z) = s (candidates for the extrema of sigma(z) - s z)."""
    if act == "relu":
        return [torch.zeros_like(s)]
    ok = (s > 0) & (s <= 1)
    zc = torch.atanh(torch.sqrt(torch.clamp(1 - s, 0.0, 1.0 - 1e-16)))
    zc = torch.where(ok, zc, torch.full_like(s, float("nan")))
    return [zc, -zc]


def _intercept(act: str, s: torch.Tensor, l: torch.Tensor, u: torch.Tensor, want_max: bool) -> torch.Tensor:
    """Exact min (or max) of sigma(z) - s z over [l, u]: endpoints and critical points inside [l, u].

    Critical points enter detached (envelope theorem: d/ds = -z*), endpoints carry their gradient."""
    cands = [act_fn(act, l) - s * l, act_fn(act, u) - s * u]
    for zc in _critical_points(act, s.detach()):
        zc = zc.detach()
        inside = (zc >= l) & (zc <= u) & ~torch.isnan(zc)
        v = act_fn(act, torch.nan_to_num(zc)) - s * torch.nan_to_num(zc)
        fill = torch.full_like(v, -math.inf if want_max else math.inf)
        cands.append(torch.where(inside, v, fill))
    C = torch.stack(cands)
    return C.max(dim=0).values if want_max else C.min(dim=0).values


def relax(act: str, l: torch.Tensor, u: torch.Tensor):
    """Per-neuron lines sL z + tL <= sigma(z) <= sU z + tU valid on [l, u]."""
    if act == "relu":
        stable_on = l >= 0
        stable_off = u <= 0
        width = torch.where(u > l, u - l, torch.ones_like(u))
        chord = torch.where(stable_on, torch.ones_like(u), torch.where(stable_off, torch.zeros_like(u), u / width))
        sU = chord
        sL = torch.where(stable_on, torch.ones_like(u),
                         torch.where(stable_off, torch.zeros_like(u),
                                     (u >= -l).to(u.dtype)))
    else:
        t_l, t_u = torch.tanh(l), torch.tanh(u)
        same = (u - l) <= 0
        width = torch.where(same, torch.ones_like(u), u - l)
        chord = torch.where(same, 1 - t_l ** 2, (t_u - t_l) / width)
        mid_slope = 1 - torch.tanh(0.5 * (l + u)) ** 2
        pos = l >= 0
        neg = u <= 0
        cross = ~pos & ~neg
        # crossing zero: tangent lines through the endpoints
        l_safe = torch.where(cross, l, -torch.ones_like(l))
        u_safe = torch.where(cross, u, torch.ones_like(u))
        d_up = _tanh_tangent_from(l_safe)                 # upper line touches at d_up > 0
        d_lo = -_tanh_tangent_from(-u_safe)               # lower line touches at d_lo < 0
        sU_cross = torch.where(d_up >= u_safe, chord, 1 - torch.tanh(d_up) ** 2)
        sL_cross = torch.where(d_lo <= l_safe, chord, 1 - torch.tanh(d_lo) ** 2)
        sU = torch.where(pos, mid_slope, torch.where(neg, chord, sU_cross))
        sL = torch.where(pos, chord, torch.where(neg, mid_slope, sL_cross))
        sU = torch.where(same, chord, sU)
        sL = torch.where(same, chord, sL)
    tL = _intercept(act, sL, l, u, want_max=False)
    tU = _intercept(act, sU, l, u, want_max=True)
    return sL, tL, sU, tU


# ------------------------------------------------------------------------------------------------
# CROWN back-substitution (Thm. 2)
# ------------------------------------------------------------------------------------------------
def _back_substitute(Ws, bs, relaxations, layer: int, upper: bool, c, r, G=None):
    """Affine bound of the pre-activation of ``layer`` (0-based index into Ws) over the box (c, r), or
    over the zonotope c + G xi, |xi|_inf <= 1, when G is given.

    Returns (Lambda, bias, value): Lambda alpha + bias bounds the layer from below (or above), and
    value is its minimum (or maximum) over the set: Lambda c -+ |Lambda| r over the box,
    Lambda c -+ ||Lambda G||_{1,r} over the zonotope."""
    Lam = Ws[layer].clone()
    bias = bs[layer].clone()
    for k in range(layer - 1, -1, -1):
        sL, tL, sU, tU = relaxations[k]
        pos = Lam >= 0
        if upper:
            s_sel = torch.where(pos, sU, sL)
            t_sel = torch.where(pos, tU, tL)
        else:
            s_sel = torch.where(pos, sL, sU)
            t_sel = torch.where(pos, tL, tU)
        # a coefficient exactly 0 contributes nothing either way; the lower line is taken for it
        zero = Lam == 0
        s_sel = torch.where(zero, sL.expand_as(Lam), s_sel)
        t_sel = torch.where(zero, tL.expand_as(Lam), t_sel)
        bias = bias + (Lam * t_sel).sum(dim=1)
        LamS = Lam * s_sel
        bias = bias + LamS @ bs[k]
        Lam = LamS @ Ws[k]
    spread = Lam.abs() @ r if G is None else (Lam @ G).abs().sum(dim=-1)
    value = Lam @ c + spread + bias if upper else Lam @ c - spread + bias
    return Lam, bias, value


def ibp_layer(W, b, act: str, l_prev, u_prev):
    """Interval bound propagation through one hidden layer: the activation is monotone, so the previous
    layer's outputs lie in [act(l), act(u)], and the affine map's range over that box is its centre
    image plus |W| times its radius."""
    hl, hh = act_fn(act, l_prev), act_fn(act, u_prev)
    hc, hr = 0.5 * (hl + hh), 0.5 * (hh - hl)
    return W @ hc - W.abs() @ hr + b, W @ hc + W.abs() @ hr + b


def crown(Ws, bs, act: str, lo: torch.Tensor, hi: torch.Tensor, intermediate: str = "crown"):
    """Thm. 2 over the box [lo, hi]: returns (W_lo, b_lo, W_hi, b_hi, hidden bounds [(l_i, u_i)]).

    ``intermediate`` selects how the pre-activation bounds of hidden layers 2.. are obtained: "crown"
    (full back-substitution, the default) or "ibp" (interval bound propagation from the previous layer's
    bounds, the cheaper and looser variant); the output layer is always back-substituted."""
    c = 0.5 * (lo + hi)
    r = 0.5 * (hi - lo)
    L = len(Ws)
    bounds = []
    relaxations = []
    l1 = Ws[0] @ c - Ws[0].abs() @ r + bs[0]
    u1 = Ws[0] @ c + Ws[0].abs() @ r + bs[0]
    bounds.append((l1, u1))
    relaxations.append(relax(act, l1, u1))
    for layer in range(1, L - 1):
        if intermediate == "ibp":
            li, ui = ibp_layer(Ws[layer], bs[layer], act, *bounds[-1])
        else:
            _, _, li = _back_substitute(Ws, bs, relaxations, layer, False, c, r)
            _, _, ui = _back_substitute(Ws, bs, relaxations, layer, True, c, r)
        bounds.append((li, ui))
        relaxations.append(relax(act, li, ui))
    W_lo, b_lo, _ = _back_substitute(Ws, bs, relaxations, L - 1, False, c, r)
    W_hi, b_hi, _ = _back_substitute(Ws, bs, relaxations, L - 1, True, c, r)
    return W_lo, b_lo, W_hi, b_hi, bounds


def remainder_bounds(Ws, bs, act: str, nominal: torch.Tensor, lo: torch.Tensor, hi: torch.Tensor,
                     residual: bool = True, intermediate: str = "crown"):
    """Thm. 3 for the dynamics x+ = [x +] MLP([x; u]). Returns (r_lo, r_hi, J_full, crown_parts).

    J_full is [A B] of the full dynamics; with ``residual`` both the CROWN slopes and J carry the same
    identity block, which therefore cancels in W - J."""
    W_lo, b_lo, W_hi, b_hi, bounds = crown(Ws, bs, act, lo, hi, intermediate)
    J = jacobian(Ws, bs, act, nominal)
    f_nom, _ = forward(Ws, bs, act, nominal)
    n_x = J.shape[0]
    if residual:
        eye = torch.zeros_like(J)
        eye[:, :n_x] = torch.eye(n_x, dtype=J.dtype)
        J = J + eye
        W_lo = W_lo + eye
        W_hi = W_hi + eye
        f_nom = f_nom + nominal[:n_x]
    c = 0.5 * (lo + hi)
    r = 0.5 * (hi - lo)
    M_lo = W_lo - J
    M_hi = W_hi - J
    const = J @ nominal - f_nom
    r_lo = M_lo @ c - M_lo.abs() @ r + const + b_lo
    r_hi = M_hi @ c + M_hi.abs() @ r + const + b_hi
    return r_lo, r_hi, J, dict(W_lo=W_lo, b_lo=b_lo, W_hi=W_hi, b_hi=b_hi, bounds=bounds)


def to_t(x) -> torch.Tensor:
    return torch.as_tensor(x, dtype=F64)


def _box_hull(a, rho, center):
    """The box center +- rho hulled with the nominal a (the set of Thm. 3 must contain it; Sec. V-A's tube
    is centred off the nominal): [min(c - rho, a), max(c + rho, a)]; the box a +- rho without a centre."""
    if center is None:
        return a - rho, a + rho
    return torch.minimum(center - rho, a), torch.maximum(center + rho, a)


def box_remainder(Ws, bs, act, x_nom, u_nom, radii, residual=True, intermediate="crown", center=None):
    """One timestep with a box set (centred at the nominal, or at ``center`` and hulled with the nominal):
    Thm. 3 bounds and [A B]. FP64 numpy out."""
    Ws_t = [to_t(W) for W in Ws]
    bs_t = [to_t(b) for b in bs]
    a = torch.cat([to_t(x_nom), to_t(u_nom)])
    rho = to_t(radii)
    with torch.no_grad():
        lo, hi = _box_hull(a, rho, None if center is None else to_t(center))
        r_lo, r_hi, J, _ = remainder_bounds(Ws_t, bs_t, act, a, lo, hi, residual, intermediate)
    return r_lo.numpy(), r_hi.numpy(), J.numpy()


def box_remainder_vjp(Ws, bs, act, x_nom, u_nom, radii, g_lo, g_hi, residual=True, center=None):
    """Gradient of sum(g_lo * r_lo + g_hi * r_hi) w.r.t. (x~, u~, radii) for a box set at the nominal, and
    also w.r.t. the centre for a box set at ``center`` (then a 4-tuple)."""
    Ws_t = [to_t(W) for W in Ws]
    bs_t = [to_t(b) for b in bs]
    x = to_t(x_nom).requires_grad_(True)
    u = to_t(u_nom).requires_grad_(True)
    rho = to_t(radii).requires_grad_(True)
    c = None if center is None else to_t(center).requires_grad_(True)
    a = torch.cat([x, u])
    lo, hi = _box_hull(a, rho, c)
    r_lo, r_hi, _, _ = remainder_bounds(Ws_t, bs_t, act, a, lo, hi, residual)
    L = (to_t(g_lo) * r_lo).sum() + (to_t(g_hi) * r_hi).sum()
    if c is None:
        gx, gu, gr = torch.autograd.grad(L, [x, u, rho])
        return gx.numpy(), gu.numpy(), gr.numpy()
    gx, gu, gr, gc = torch.autograd.grad(L, [x, u, rho, c])
    return gx.numpy(), gu.numpy(), gr.numpy(), gc.numpy()


def zono_hull_remainder_vjp(Ws, bs, act, x_nom, u_nom, G, g_lo, g_hi, residual=True, center=None):
    """Gradient of sum(g_lo * r_lo + g_hi * r_hi) w.r.t. (x~, u~, G[, centre]) for a zonotope set taken as its
    interval hull (Eq. 21): the box of half-widths sum_g |G_ig| around the centre (the nominal without one),
    hulled with the nominal, then Thm. 3 over that box."""
    Ws_t = [to_t(W) for W in Ws]
    bs_t = [to_t(b) for b in bs]
    x = to_t(x_nom).requires_grad_(True)
    u = to_t(u_nom).requires_grad_(True)
    Gt = to_t(G).requires_grad_(True)
    c = None if center is None else to_t(center).requires_grad_(True)
    a = torch.cat([x, u])
    lo, hi = _box_hull(a, Gt.abs().sum(dim=1), c)
    r_lo, r_hi, _, _ = remainder_bounds(Ws_t, bs_t, act, a, lo, hi, residual)
    L = (to_t(g_lo) * r_lo).sum() + (to_t(g_hi) * r_hi).sum()
    if c is None:
        gx, gu, gG = torch.autograd.grad(L, [x, u, Gt])
        return gx.numpy(), gu.numpy(), gG.numpy()
    gx, gu, gG, gc = torch.autograd.grad(L, [x, u, Gt, c])
    return gx.numpy(), gu.numpy(), gG.numpy(), gc.numpy()


def zono_hull_nominal(nominal: torch.Tensor, c: torch.Tensor, G: torch.Tensor):
    """A zonotope that contains both c + G E and the nominal point: the segment from c to the nominal
    appended as one more generator, (c + a) / 2 + [G, (a - c) / 2] E (the set itself when c = a)."""
    half = 0.5 * (nominal - c)
    return c + half, torch.cat([G, half[:, None]], dim=1)


def crown_zono(Ws, bs, act: str, c: torch.Tensor, G: torch.Tensor):
    """Thm. 2 over the zonotope c + G E: the same back-substitution and relaxations as ``crown``, every
    bound concretised over the zonotope instead of its interval hull."""
    L = len(Ws)
    bounds = []
    relaxations = []
    spread = (Ws[0] @ G).abs().sum(dim=1)
    l1 = Ws[0] @ c - spread + bs[0]
    u1 = Ws[0] @ c + spread + bs[0]
    bounds.append((l1, u1))
    relaxations.append(relax(act, l1, u1))
    for layer in range(1, L - 1):
        _, _, li = _back_substitute(Ws, bs, relaxations, layer, False, c, None, G)
        _, _, ui = _back_substitute(Ws, bs, relaxations, layer, True, c, None, G)
        bounds.append((li, ui))
        relaxations.append(relax(act, li, ui))
    W_lo, b_lo, _ = _back_substitute(Ws, bs, relaxations, L - 1, False, c, None, G)
    W_hi, b_hi, _ = _back_substitute(Ws, bs, relaxations, L - 1, True, c, None, G)
    return W_lo, b_lo, W_hi, b_hi, bounds


def zono_remainder(Ws, bs, act, x_nom, u_nom, G, center=None, residual=True):
    """Thm. 3 over a zonotope tube set (Eq. 18a) concretised exactly: the set hulled with the nominal
    (``zono_hull_nominal``), CROWN over it, and r = min / max over the zonotope of the affine remainder
    bounds, M c -+ ||M G||_{1,r} + const. FP64 numpy out: (r_lo, r_hi, [A B])."""
    Ws_t = [to_t(W) for W in Ws]
    bs_t = [to_t(b) for b in bs]
    a = torch.cat([to_t(x_nom), to_t(u_nom)])
    c0 = a if center is None else to_t(center)
    with torch.no_grad():
        c, Gh = zono_hull_nominal(a, c0, to_t(G))
        W_lo, b_lo, W_hi, b_hi, _ = crown_zono(Ws_t, bs_t, act, c, Gh)
        J = jacobian(Ws_t, bs_t, act, a)
        f_nom, _ = forward(Ws_t, bs_t, act, a)
        n_x = J.shape[0]
        if residual:
            eye = torch.zeros_like(J)
            eye[:, :n_x] = torch.eye(n_x, dtype=J.dtype)
            J = J + eye
            W_lo = W_lo + eye
            W_hi = W_hi + eye
            f_nom = f_nom + a[:n_x]
        const = J @ a - f_nom
        M_lo, M_hi = W_lo - J, W_hi - J
        r_lo = M_lo @ c - (M_lo @ Gh).abs().sum(dim=1) + const + b_lo
        r_hi = M_hi @ c + (M_hi @ Gh).abs().sum(dim=1) + const + b_hi
    return r_lo.numpy(), r_hi.numpy(), J.numpy()
