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
