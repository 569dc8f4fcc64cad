"""A-priori rounding analysis of CROWN back-substitution with reduced-precision GEMM operands, FP64.

Test infrastructure: only tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline use it.
It is not the paper's method (the paper does not fix a precision, Sec. IV-D); it restates the standard
forward error analysis of a dot product (Higham, "Accuracy and Stability of Numerical Algorithms",
Sec. 3.1: |fl(x^T y) - x^T y| <= gamma_K |x|^T |y| with gamma_K = K u / (1 - K u)) for the chain of
Thm. 2 when every stage Lambda' = (Lambda o s) W_k rounds its operand a = Lambda o s to a reduced format
(FP16 or BF16, unit roundoff u_op; the product itself is first rounded to FP32), uses weights W~ rounded
to the same format and accumulates in FP32 (unit roundoff 2^-23 here: no round-to-nearest assumed).

With a~ = fl(a) and W~ = fl(W), the computed stage differs from the exact (Lambda o s) W_k by at most
    gamma_K |a~| |W~| + |a~ - a| |W~| + |a| |W~ - W|,
and since the next stage sees that error only through Lambda' dh_{k-1}, with |dh_{k-1}| <= abar_{k-1}
over the set (abar = max |sigma(z) - sigma(z~)|, the input radius for k = 0), the bound moves by at most
    sum_j |a_j| w_j,   w_j = c1 (|W~| abar)_j + (|W - W~| abar)_j,   c1 = u_op + 2^-24 + gamma_K (1 + u_op),
plus u_sub (1 + gamma_K) sum_j (|W~| abar)_j for operands that round into the subnormal range (u_sub =
half the format's smallest subnormal). Summed over the stages of a chain, this is the inflation a sound
reduced-precision bound must subtract (add, for upper bounds).

The functions here compute that figure on the oracle's own FP64 Lambda chains (``crown.py``) and an
envelope of what a kernel that applies it can return: the same CROWN algorithm with every hidden layer's
bounds widened by ``k`` times their inflation and the output bounds moved by ``k`` times theirs. k = 1
models a kernel whose arithmetic happens to be exact; k = 2 covers any actual rounding error up to the
a-priori bound (the computed value lies within one inflation of the exact one, and the kernel subtracts
one more). Hidden layer 1's bounds are not back-substituted (exact interval product), so they carry no
inflation.
"""
from __future__ import annotations

import torch

from . import crown

F64 = torch.float64
FORMATS = {
    # unit roundoff, half the smallest positive subnormal
    "fp16": (2.0 ** -11, 2.0 ** -25),
    "bf16": (2.0 ** -8, 2.0 ** -134),
    # FP32 operands: the only operand rounding is that of the product Lambda o s itself
    "fp32": (2.0 ** -24, 2.0 ** -150),
}


def round_to(x: torch.Tensor, fmt: str) -> torch.Tensor:
    """Round-to-nearest-even into FP16 / BF16, back in FP64 (FP64 -> FP32 first, as an FP32 value is what
    gets rounded)."""
    dt = {"fp16": torch.float16, "bf16": torch.bfloat16, "fp32": torch.float32}[fmt]
    return x.to(torch.float32).to(dt).to(F64)


def gamma(K: int, u: float = 2.0 ** -23) -> float:
    return K * u / (1.0 - K * u)


def stage_weights(W: torch.Tensor, abar_prev: torch.Tensor, fmt: str):
    """Per-neuron inflation weight w and the per-stage constant of the stage that multiplies by W
    ([K, N]: K neurons of the operand, N of the next layer down), given abar of the layer below."""
    u_op, u_sub = FORMATS[fmt]
    K = W.shape[0]
    g = gamma(K)
    Wt = round_to(W, fmt)
    v1 = Wt.abs() @ abar_prev
    v2 = (W - Wt).abs() @ abar_prev
    c1 = u_op + 2.0 ** -24 + g * (1.0 + u_op)
    w = c1 * v1 + v2
    const = u_sub * (1.0 + g) * float(v1.sum())
    return w, const


def _abar(act: str, l: torch.Tensor, u: torch.Tensor, z_nom: torch.Tensor) -> torch.Tensor:
    """Bound on |sigma(z) - sigma(z~)| over z in [l, u] (sigma monotone)."""
    s = lambda z: crown.act_fn(act, z)
    return torch.maximum((s(u) - s(z_nom)).abs(), (s(z_nom) - s(l)).abs())


def _chain(Ws, relaxations, layer: int, upper: bool, weights):
    """Back-substitution from the rows of ``layer`` (the oracle's line selection) with the inflation of
    every stage accumulated per row. Returns (Lambda over the input, inflation per row)."""
    Lam = Ws[layer].clone()
    infl = torch.zeros(Lam.shape[0], dtype=F64)
    for k in range(layer - 1, -1, -1):
        sL, tL, sU, tU = relaxations[k]
        pos = Lam >= 0
        s_sel = torch.where(pos, sU, sL) if upper else torch.where(pos, sL, sU)
        s_sel = torch.where(Lam == 0, sL.expand_as(Lam), s_sel)
        a = Lam * s_sel
        w, const = weights[k]
        infl = infl + a.abs() @ w + const
        Lam = a @ Ws[k]
    return Lam, infl


def crown_envelope(Ws, bs, act: str, nominal: torch.Tensor, lo: torch.Tensor, hi: torch.Tensor, fmt: str,
                   k: float):
    """CROWN (Thm. 2) over the box [lo, hi] with the reduced-precision inflation applied k times to every
    back-substituted bound. Returns (W_lo, b_lo, W_hi, b_hi, infl_lo, infl_hi, bounds) where infl_* is the
    output chains' inflation (one times) and bounds the widened hidden-layer bounds."""
    c = 0.5 * (lo + hi)
    r = 0.5 * (hi - lo)
    _, z_nom = crown.forward(Ws, bs, act, nominal)
    L = len(Ws)
    abar_in = torch.maximum((hi - nominal).abs(), (nominal - lo).abs())
    weights = [stage_weights(Ws[0], abar_in, fmt)]
    l1 = Ws[0] @ c - Ws[0].abs() @ r + bs[0]
    u1 = Ws[0] @ c + Ws[0].abs() @ r + bs[0]
    bounds = [(l1, u1)]
    relaxations = [crown.relax(act, l1, u1)]
    for layer in range(1, L - 1):
        weights.append(stage_weights(Ws[layer], _abar(act, *bounds[-1], z_nom[layer - 1]), fmt))
        _, _, li = crown._back_substitute(Ws, bs, relaxations, layer, False, c, r)
        _, _, ui = crown._back_substitute(Ws, bs, relaxations, layer, True, c, r)
        _, il = _chain(Ws, relaxations, layer, False, weights)
        _, iu = _chain(Ws, relaxations, layer, True, weights)
        li, ui = li - k * il, ui + k * iu
        bounds.append((li, ui))
        relaxations.append(crown.relax(act, li, ui))
    weights.append(None)   # the output layer is never an operand
    W_lo, b_lo, _ = crown._back_substitute(Ws, bs, relaxations, L - 1, False, c, r)
    W_hi, b_hi, _ = crown._back_substitute(Ws, bs, relaxations, L - 1, True, c, r)
    _, il = _chain(Ws, relaxations, L - 1, False, weights)
    _, iu = _chain(Ws, relaxations, L - 1, True, weights)
    return W_lo, b_lo, W_hi, b_hi, il, iu, bounds


def remainder_envelope(Ws, bs, act: str, x_nom, u_nom, radii, fmt: str, k: float, residual: bool = True):
    """Thm. 3 on ``crown_envelope`` for one timestep with a box set centred at the nominal: returns FP64
    numpy (r_lo, r_hi, infl_lo, infl_hi) with r_lo = the Thm. 3 lower bound - k infl_lo (r_hi likewise)
    and infl_* the output chains' inflation (one times)."""
    Ws_t = [crown.to_t(W) for W in Ws]
    bs_t = [crown.to_t(b) for b in bs]
    a = torch.cat([crown.to_t(x_nom), crown.to_t(u_nom)])
    rho = crown.to_t(radii)
    lo, hi = a - rho, a + rho
    with torch.no_grad():
        W_lo, b_lo, W_hi, b_hi, il, iu, _ = crown_envelope(Ws_t, bs_t, act, a, lo, hi, fmt, k)
        J = crown.jacobian(Ws_t, bs_t, act, a)
        f_nom, _ = crown.forward(Ws_t, bs_t, act, a)
        # the residual identity cancels in W - J (it is exact in both)
        c = 0.5 * (lo + hi)
        r = 0.5 * (hi - lo)
        const = J @ a - f_nom
        M_lo, M_hi = W_lo - J, W_hi - J
        r_lo = M_lo @ c - M_lo.abs() @ r + const + b_lo - k * il
        r_hi = M_hi @ c + M_hi.abs() @ r + const + b_hi + k * iu
    return r_lo.numpy(), r_hi.numpy(), il.numpy(), iu.numpy()


def stage_error_bound(a: torch.Tensor, W: torch.Tensor, fmt: str) -> torch.Tensor:
    """Entrywise bound on |computed - a W| for one stage (a: [R, K] FP64 operand rows, W: [K, N]): the
    analysis above before it is multiplied by abar, sum_j |a_j| (c1 |W~_j.| + |W_j. - W~_j.|) + the
    subnormal term."""
    u_op, u_sub = FORMATS[fmt]
    g = gamma(W.shape[0])
    Wt = round_to(W, fmt)
    c1 = u_op + 2.0 ** -24 + g * (1.0 + u_op)
    return a.abs() @ (c1 * Wt.abs() + (W - Wt).abs()) + u_sub * (1.0 + g) * Wt.abs().sum(dim=0)


def emulate_stage(a: torch.Tensor, W: torch.Tensor, fmt: str) -> torch.Tensor:
    """One stage computed the way a reduced-precision kernel computes it: the operand rounded to FP32 and
    then to the format, the weights rounded to the format, the products summed in FP32 (torch's FP32
    matmul of the rounded values). Checks the analysis against an actual rounded computation."""
    at = round_to(a, fmt).to(torch.float32)
    return (at @ round_to(W, fmt).to(torch.float32)).to(F64)


def unit_roundoff(fmt: str) -> float:
    return FORMATS[fmt][0]


def jacobian_error_bound(Ws, bs, act: str, nominal, fmt: str):
    """Elementwise a-priori bound on |J~ - J| for the Jacobian chain J = W_L D_{L-1} ... D_1 W_1 computed
    like the bound chains (operand W_L o sigma', then (Lambda o sigma') W_k per stage, each stage as in the
    analysis above). To first order in the unit roundoffs, stage k's relative error (2 u_op + 2^-24 +
    gamma_K, operand and weight rounding plus FP32 sums) carries through the exact remaining stages, which
    are bounded in magnitude by the absolute chain M = |W_L| |D_{L-1}| ... |D_1| |W_1|; the sum over the
    L - 1 stages, times 1.01 for the second-order terms, bounds the error. FP64 numpy [n_x, n]."""
    Ws_t = [crown.to_t(W) for W in Ws]
    bs_t = [crown.to_t(b) for b in bs]
    a = crown.to_t(nominal)
    u_op, _ = FORMATS[fmt]
    with torch.no_grad():
        _, zs = crown.forward(Ws_t, bs_t, act, a)
        M = Ws_t[-1].abs()
        rel = 0.0
        for k in range(len(Ws_t) - 2, -1, -1):
            M = (M * crown.act_deriv(act, zs[k]).abs()) @ Ws_t[k].abs()
            rel += 2.0 * u_op + 2.0 ** -24 + gamma(Ws_t[k].shape[0])
    return (1.01 * rel * M).numpy()


def emulate_jacobian(Ws, bs, act: str, nominal, fmt: str):
    """The Jacobian chain computed with rounded operands (``emulate_stage`` per stage), FP64 numpy."""
    Ws_t = [crown.to_t(W) for W in Ws]
    bs_t = [crown.to_t(b) for b in bs]
    a = crown.to_t(nominal)
    with torch.no_grad():
        _, zs = crown.forward(Ws_t, bs_t, act, a)
        Lam = Ws_t[-1]
        for k in range(len(Ws_t) - 2, -1, -1):
            op = (Lam.to(torch.float32) * crown.act_deriv(act, zs[k]).to(torch.float32)).to(F64)
            Lam = emulate_stage(op, Ws_t[k], fmt)
    return Lam.numpy()


# ------------------------------------------------------------------------------------------------
# Zonotope sets concretised exactly (Sec. IV-C sets, Eq. 18a) with a reduced-precision last product
# ------------------------------------------------------------------------------------------------
# Over the zonotope Z = cd (1 - xi_0) + G xi (the tube set hulled with the nominal, Delta = alpha - a,
# cd = (c - a) / 2, |xi|_inf <= 1) the minimum of M Delta is V = v_0 - sum_{g >= 1} |v_g| with
# v = M [cd | G | -cd]. A kernel that forms v with M and the block rounded to the format (cd first
# rounded to FP32 from fl(c - a) / 2) and FP32 sums of K products errs on V by at most, per row,
#   sum_i |M_i| (cz h_i + wadd) + zc1 sum_i h_i + zc2
# with h_i = 2 |cd_i| + sum_g |G_ig| (the hull's half-width) and
#   cz = (gamma_K (1 + u) + u)(1 + u) + u + 2^-23,  wadd = (Pp + 2) u_sub (2 + gamma_K),
#   zc1 = u_sub (1 + u)(1 + gamma_K),                 zc2 = 2 n (Pp + 2) u_sub^2,
# Pp = n_gen + 2 rounded up to 16 (the product's columns) and K = n rounded up to 64. Derivation: with
# M~ = fl(M), B~ = fl(B), |M~ - M| <= u |M| + u_sub, |B~ - B| <= u |B| + u_sub entrywise, the error of
# every column is |M~ B~ - M B| + gamma_K |M~| |B~| <= (|M~ - M| |B~| + |M| |B~ - B|) + gamma_K |M~||B~|;
# summed over the columns with sum_g |B_ig| <= h_i (1 + 2^-24) + 2^-149 (cd's FP32 rounding, which also
# moves V itself by at most |M| (2^-24 h + 2^-149)) this gives the terms above.


def zono_stage_constants(n: int, n_gen: int, fmt: str):
    """(cz, wadd, zc1, zc2, Pp) of the zonotope stage for n inputs and n_gen generators."""
    u, u_sub = FORMATS[fmt]
    K = 64 * ((n + 63) // 64)
    g = gamma(K)
    Pp = 16 * ((n_gen + 2 + 15) // 16)
    cz = (g * (1 + u) + u) * (1 + u) + u + 2.0 ** -23
    wadd = (Pp + 2) * u_sub * (2 + g)
    zc1 = u_sub * (1 + u) * (1 + g)
    zc2 = 2.0 * n * (Pp + 2) * u_sub ** 2
    return cz, wadd, zc1, zc2, Pp


def zono_stage_allowance(M: torch.Tensor, h: torch.Tensor, n_gen: int, fmt: str) -> torch.Tensor:
    """Per-row bound on |computed V - exact V| (M: [R, n] FP64 rows, h: [n] hull half-widths)."""
    cz, wadd, zc1, zc2, _ = zono_stage_constants(M.shape[1], n_gen, fmt)
    return M.abs() @ (cz * h + wadd) + zc1 * float(h.sum()) + zc2


def zono_min(M: torch.Tensor, cd: torch.Tensor, G: torch.Tensor) -> torch.Tensor:
    """Exact min over Z of M Delta, FP64: M cd - |M cd| - sum_g |M G_g|."""
    v0 = M @ cd
    return v0 - v0.abs() - (M @ G).abs().sum(dim=1)


def emulate_zono_stage(M: torch.Tensor, c: torch.Tensor, a: torch.Tensor, G: torch.Tensor, fmt: str):
    """V computed the way a reduced-precision kernel computes it: cd = fl32(c - a) / 2, the block
    [cd | G | -cd] and M rounded to the format, the products summed in FP32 (torch's FP32 matmul)."""
    cd = ((c.to(torch.float32) - a.to(torch.float32)) * 0.5).to(F64)
    block = torch.cat([cd[:, None], G, -cd[:, None]], dim=1)
    v = (round_to(M, fmt).to(torch.float32) @ round_to(block, fmt).to(torch.float32)).to(F64)
    return v[:, 0] - v[:, 1:].abs().sum(dim=1)


def zono_remainder_envelope(Ws, bs, act: str, x_nom, u_nom, G, center, fmt: str, k: float,
                            residual: bool = True):
    """Thm. 3 over the zonotope tube set concretised exactly (``crown.zono_remainder``) with the
    reduced-precision inflation applied k times: every hidden layer's bounds (the first one included,
    which now also comes out of a rounded product) widened by k times their chain inflation plus the
    zonotope stage's allowance, and the output bounds moved by k times theirs. Returns FP64 numpy
    (r_lo, r_hi, infl_lo, infl_hi), infl_* the output rows' total inflation (one times)."""
    Ws_t = [crown.to_t(W) for W in Ws]
    bs_t = [crown.to_t(b) for b in bs]
    a = torch.cat([crown.to_t(x_nom), crown.to_t(u_nom)])
    G0 = crown.to_t(G)
    c0 = a if center is None else crown.to_t(center)
    n_gen = G0.shape[1]
    with torch.no_grad():
        c, Gh = crown.zono_hull_nominal(a, c0, G0)
        h = Gh.abs().sum(dim=1) + (c - a).abs()                 # the hull's half-width around a
        allow = lambda M: zono_stage_allowance(M, h, n_gen, fmt)
        _, z_nom = crown.forward(Ws_t, bs_t, act, a)
        L = len(Ws_t)
        weights = [stage_weights(Ws_t[0], h, fmt)]
        spread = (Ws_t[0] @ Gh).abs().sum(dim=1)
        a0 = allow(Ws_t[0])
        l1 = Ws_t[0] @ c - spread + bs_t[0] - k * a0
        u1 = Ws_t[0] @ c + spread + bs_t[0] + k * a0
        bounds = [(l1, u1)]
        relaxations = [crown.relax(act, l1, u1)]
        for layer in range(1, L - 1):
            weights.append(stage_weights(Ws_t[layer], _abar(act, *bounds[-1], z_nom[layer - 1]), fmt))
            Ll, _, li = crown._back_substitute(Ws_t, bs_t, relaxations, layer, False, c, None, Gh)
            Lu, _, ui = crown._back_substitute(Ws_t, bs_t, relaxations, layer, True, c, None, Gh)
            _, il = _chain(Ws_t, relaxations, layer, False, weights)
            _, iu = _chain(Ws_t, relaxations, layer, True, weights)
            li, ui = li - k * (il + allow(Ll)), ui + k * (iu + allow(Lu))
            bounds.append((li, ui))
            relaxations.append(crown.relax(act, li, ui))
        weights.append(None)
        W_lo, b_lo, _ = crown._back_substitute(Ws_t, bs_t, relaxations, L - 1, False, c, None, Gh)
        W_hi, b_hi, _ = crown._back_substitute(Ws_t, bs_t, relaxations, L - 1, True, c, None, Gh)
        _, il = _chain(Ws_t, relaxations, L - 1, False, weights)
        _, iu = _chain(Ws_t, relaxations, L - 1, True, weights)
        J = crown.jacobian(Ws_t, bs_t, act, a)
        f_nom, _ = crown.forward(Ws_t, bs_t, act, a)
        const = J @ a - f_nom           # the residual identity cancels in W - J
        M_lo, M_hi = W_lo - J, W_hi - J
        il = il + allow(M_lo)
        iu = iu + allow(M_hi)
        r_lo = M_lo @ c - (M_lo @ Gh).abs().sum(dim=1) + const + b_lo - k * il
        r_hi = M_hi @ c + (M_hi @ Gh).abs().sum(dim=1) + const + b_hi + k * iu
    return r_lo.numpy(), r_hi.numpy(), il.numpy(), iu.numpy()
