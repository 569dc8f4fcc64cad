"""Pins of the FP64 CROWN oracle (Thms. 2-3) and the proposer oracle (CPU only)."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import crown, exact, proposer, sampling
from paper_2607_01203_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
T64 = torch.float64


def _net(widths, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    Ws = [rng.normal(size=(o, i)) * scale / math.sqrt(i) for i, o in zip(widths[:-1], widths[1:])]
    bs = [rng.normal(size=o) * 0.1 for o in widths[1:]]
    return Ws, bs


def test_worked_examples_golden():
    """Hand-derived Thm. 2/3 values for two scalar ReLU nets (tests/golden/crown_worked_examples.txt)."""
    rows = {}
    with open(os.path.join(GOLDEN, "crown_worked_examples.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                p = line.split()
                rows[p[0]] = [float(v) for v in p[1:]]
    one = torch.ones(1, 1, dtype=T64)
    nets = {"A": ([one, one], [torch.zeros(1, dtype=T64)] * 2, 0.5),
            "B": ([one, one, one], [torch.zeros(1, dtype=T64), torch.tensor([-0.5], dtype=T64),
                                    torch.zeros(1, dtype=T64)], 1.5)}
    lo = torch.tensor([-1.0], dtype=T64)
    hi = torch.tensor([2.0], dtype=T64)
    for name, (Ws, bs, a) in nets.items():
        g = rows[name]
        r_lo, r_hi, J, parts = crown.remainder_bounds(Ws, bs, "relu", torch.tensor([a], dtype=T64), lo, hi,
                                                      residual=False)
        got = [parts["W_lo"].item(), parts["b_lo"].item(), parts["W_hi"].item(), parts["b_hi"].item(),
               r_lo.item(), r_hi.item()]
        assert got == pytest.approx(g[:6], abs=1e-14)
        el, eh, _ = exact.relu_exact_range([W.numpy() for W in Ws], [b.numpy() for b in bs], np.array([a]),
                                           lo.numpy(), hi.numpy(), residual=False)
        assert el[0] == pytest.approx(g[6], abs=1e-12) and eh[0] == pytest.approx(g[7], abs=1e-12)


@pytest.mark.parametrize("act", ["relu", "tanh"])
def test_relaxation_lines_valid(act):
    """sL z + tL <= sigma(z) <= sU z + tU on [l, u], for crossing, one-sided and degenerate intervals."""
    rng = np.random.default_rng(6)
    l = rng.normal(size=400) * 2
    u = l + np.abs(rng.normal(size=400)) * rng.choice([0.0, 0.01, 1, 4], size=400)
    lt, ut = torch.tensor(l, dtype=T64), torch.tensor(u, dtype=T64)
    sL, tL, sU, tU = crown.relax(act, lt, ut)
    z = lt[None, :] + torch.linspace(0, 1, 2001, dtype=T64)[:, None] * (ut - lt)[None, :]
    s = crown.act_fn(act, z)
    assert torch.all(sL * z + tL <= s + 1e-13)
    assert torch.all(sU * z + tU >= s - 1e-13)
    # lines touch the function (intercepts are exact extrema, not slack)
    gapL = (s - (sL * z + tL)).min(dim=0).values
    gapU = ((sU * z + tU) - s).min(dim=0).values
    assert gapL.max() < 1e-6 and gapU.max() < 1e-6


def test_tanh_slope_rules_closed_form():
    """l >= 0: upper tangent at the midpoint, lower chord (textbook concave case)."""
    l, u = torch.tensor([0.0], dtype=T64), torch.tensor([1.0], dtype=T64)
    sL, tL, sU, tU = crown.relax("tanh", l, u)
    assert sL.item() == pytest.approx(math.tanh(1.0), abs=1e-15) and tL.item() == pytest.approx(0.0, abs=1e-15)
    s_mid = 1 - math.tanh(0.5) ** 2
    assert sU.item() == pytest.approx(s_mid, abs=1e-15)
    assert tU.item() == pytest.approx(math.tanh(0.5) - s_mid * 0.5, abs=1e-12)


def test_crown_affine_bounds_hold():
    """Thm. 2's statement: W_lo a + b_lo <= f(a) <= W_hi a + b_hi for sampled a in the box."""
    rng = np.random.default_rng(7)
    for act in ("relu", "tanh"):
        Ws, bs = _net((6, 16, 16, 16, 4), 8)
        Wt = [torch.tensor(W) for W in Ws]
        bt = [torch.tensor(b) for b in bs]
        a = rng.normal(size=6)
        lo, hi = a - 0.3, a + 0.3
        W_lo, b_lo, W_hi, b_hi, _ = crown.crown(Wt, bt, act, torch.tensor(lo), torch.tensor(hi))
        P = sampling.box_points(lo, hi, 30000, rng)
        F = sampling.mlp_f_batch(Ws, bs, act, residual=False)(P)
        assert np.all(P @ W_lo.numpy().T + b_lo.numpy() <= F + 1e-12)
        assert np.all(P @ W_hi.numpy().T + b_hi.numpy() >= F - 1e-12)


def test_jacobian_matches_finite_differences():
    Ws, bs = _net((5, 12, 12, 3), 9)
    Wt = [torch.tensor(W) for W in Ws]
    bt = [torch.tensor(b) for b in bs]
    a = torch.tensor(np.random.default_rng(10).normal(size=5))
    J = crown.jacobian(Wt, bt, "tanh", a).numpy()
    f = lambda x: crown.forward(Wt, bt, "tanh", torch.tensor(x))[0].numpy()
    Jfd = np.stack([(f(a.numpy() + e) - f(a.numpy() - e)) / 2e-6 for e in np.eye(5) * 1e-6], axis=1)
    assert np.abs(J - Jfd).max() < 1e-8


def test_relu_contains_exact_range_workload():
    """Thm. 3 soundness on the 8->64->64->6 workload: CROWN contains the enumerated exact range."""
    w = inputs.relu_mlp()
    for t in (0, 9, 19):
        a = w.nominal()[t].astype(np.float64)
        r_lo, r_hi, J = crown.box_remainder(w.Ws, w.bs, "relu", w.x_nom[t], w.u_nom[t], w.radii[t])
        el, eh, nreg = exact.relu_exact_range(w.Ws, w.bs, a, a - w.radii[t], a + w.radii[t])
        assert nreg >= 1
        assert np.all(r_lo <= el + 1e-12) and np.all(r_hi >= eh - 1e-12)


def test_relu_small_net_exact_and_enumeration_cross_check():
    """2->4->4->2 net: enumeration agrees with dense brute force; CROWN contains both."""
    Ws, bs = _net((2, 4, 4, 2), 11, scale=1.5)
    a = np.array([0.1, -0.2])
    lo, hi = a - 0.4, a + 0.4
    el, eh, nreg = exact.relu_exact_range(Ws, bs, a, lo, hi, residual=False)
    g = np.linspace(0, 1, 401)
    P = np.stack(np.meshgrid(lo[0] + g * 0.8, lo[1] + g * 0.8), -1).reshape(-1, 2)
    Wt = [torch.tensor(W) for W in Ws]
    bt = [torch.tensor(b) for b in bs]
    J = crown.jacobian(Wt, bt, "relu", torch.tensor(a)).numpy()
    R = sampling.remainders(sampling.mlp_f_batch(Ws, bs, "relu", residual=False), a, J, P)
    assert np.allclose(R.min(0), el, atol=5e-3) and np.allclose(R.max(0), eh, atol=5e-3)
    assert np.all(R.min(0) >= el - 1e-12) and np.all(R.max(0) <= eh + 1e-12)
    r_lo, r_hi, _, _ = crown.remainder_bounds(Wt, bt, "relu", torch.tensor(a), torch.tensor(lo),
                                              torch.tensor(hi), residual=False)
    assert np.all(r_lo.numpy() <= el + 1e-12) and np.all(r_hi.numpy() >= eh - 1e-12)


def test_all_stable_relu_gives_zero():
    """An all-stable box makes f affine on X, so the exact remainder and the Thm. 3 bound are 0."""
    Ws, bs = _net((3, 8, 8, 3), 12)
    Ws = [np.abs(W) for W in Ws]                         # positive weights and biases keep every
    bs = [np.abs(b) + 5.0 for b in bs[:-1]] + [bs[-1]]  # hidden neuron active on the box
    Wt = [torch.tensor(W) for W in Ws]
    bt = [torch.tensor(b) for b in bs]
    a = torch.tensor([0.1, 0.2, -0.1], dtype=T64)
    r_lo, r_hi, _, parts = crown.remainder_bounds(Wt, bt, "relu", a, a - 0.05, a + 0.05)
    assert all(bool((l > 0).all()) for l, _ in parts["bounds"])
    assert torch.abs(r_lo).max() < 1e-13 and torch.abs(r_hi).max() < 1e-13


def test_tanh_scalar_brute_force_grid():
    """1 -> 1 -> 1 tanh net: the bound contains the remainder on a 10^6-point grid, and is near-tight."""
    Ws = [torch.tensor([[1.3]], dtype=T64), torch.tensor([[0.8]], dtype=T64)]
    bs = [torch.tensor([0.2], dtype=T64), torch.tensor([0.0], dtype=T64)]
    for a0, rad in ((0.3, 0.5), (-1.0, 0.2), (2.0, 1.0)):
        a = torch.tensor([a0], dtype=T64)
        r_lo, r_hi, J, _ = crown.remainder_bounds(Ws, bs, "tanh", a, a - rad, a + rad, residual=False)
        x = np.linspace(a0 - rad, a0 + rad, 1_000_001)
        f = 0.8 * np.tanh(1.3 * x + 0.2)
        r = f - f[500000] - J.item() * (x - a0)
        assert r.min() >= r_lo.item() - 1e-12 and r.max() <= r_hi.item() + 1e-12
        assert (r_hi - r_lo).item() <= 4.0 * (r.max() - r.min())


def test_tanh_linear_limit_and_sampling():
    """Near-linear net (tiny weights): width vanishes like scale^3; the workload net is sound by sampling."""
    widths = (6, 16, 16, 3)
    widths_prev = None
    for scale in (0.1, 0.01):
        Ws, bs = _net(widths, 13, scale=scale)
        Wt = [torch.tensor(W) for W in Ws]
        bt = [torch.tensor(b) * 0 for b in bs]
        a = torch.zeros(6, dtype=T64)
        r_lo, r_hi, _, _ = crown.remainder_bounds(Wt, bt, "tanh", a, a - 0.5, a + 0.5, residual=False)
        wdt = (r_hi - r_lo).max().item()
        if widths_prev is not None:
            assert wdt < widths_prev * 2e-3
        widths_prev = wdt
    w = inputs.tanh_mlp(n_traj=1, N=3)
    rng = np.random.default_rng(14)
    for t in range(3):
        a = w.nominal()[t].astype(np.float64)
        r_lo, r_hi, J = crown.box_remainder(w.Ws, w.bs, "tanh", w.x_nom[t], w.u_nom[t], w.radii[t])
        P = sampling.box_points(a - w.radii[t], a + w.radii[t], 20000, rng)
        R = sampling.remainders(sampling.mlp_f_batch(w.Ws, w.bs, "tanh"), a, J, P)
        assert np.all(R >= r_lo - 1e-12) and np.all(R <= r_hi + 1e-12)


def test_oracle_gradient_matches_finite_differences():
    """The oracle's reverse-mode gradient of the bound vs central differences (h = 1e-4, FP64)."""
    w = inputs.tanh_mlp(n_traj=1, N=2, widths=(10, 16, 16, 6))
    rng = np.random.default_rng(15)
    t = 1
    x, u, rad = (w.x_nom[t].astype(np.float64), w.u_nom[t].astype(np.float64), w.radii[t].astype(np.float64))
    g_lo = rng.normal(size=6)
    g_hi = rng.normal(size=6)
    gx, gu, gr = crown.box_remainder_vjp(w.Ws, w.bs, "tanh", x, u, rad, g_lo, g_hi)

    def L(x_, u_, r_):
        lo, hi, _ = crown.box_remainder(w.Ws, w.bs, "tanh", x_, u_, r_)
        return float(g_lo @ lo + g_hi @ hi)

    h = 1e-4
    for vec, grad, which in ((x, gx, 0), (u, gu, 1), (rad, gr, 2)):
        for i in range(len(vec)):
            e = np.zeros_like(vec)
            e[i] = h
            args_p = [x, u, rad]
            args_m = [x, u, rad]
            args_p[which] = vec + e
            args_m[which] = vec - e
            fd = (L(*args_p) - L(*args_m)) / (2 * h)
            assert fd == pytest.approx(grad[i], rel=2e-3, abs=2e-6)


def test_oracle_gradient_off_centre_box_matches_finite_differences():
    """The oracle's gradient for a box centred off the nominal, hulled with it, w.r.t. (x~, u~, radii,
    centre) vs central differences (h = 1e-5, FP64). Half the coordinates have the nominal inside the box
    (|c - a| = rho / 2), half outside it (|c - a| = 2 rho: that side of the hull is the nominal itself),
    both far from the kinks at |c - a| = rho."""
    w = inputs.tanh_mlp(n_traj=1, N=2, widths=(10, 16, 16, 6))
    rng = np.random.default_rng(16)
    t = 1
    x, u, rad = (w.x_nom[t].astype(np.float64), w.u_nom[t].astype(np.float64), w.radii[t].astype(np.float64))
    a = np.concatenate([x, u])
    scale = np.where(np.arange(a.size) % 2 == 0, 0.5, 2.0) * rng.choice([-1.0, 1.0], a.size)
    c = a + scale * rad
    g_lo = rng.normal(size=6)
    g_hi = rng.normal(size=6)
    gx, gu, gr, gc = crown.box_remainder_vjp(w.Ws, w.bs, "tanh", x, u, rad, g_lo, g_hi, center=c)

    def L(x_, u_, r_, c_):
        lo, hi, _ = crown.box_remainder(w.Ws, w.bs, "tanh", x_, u_, r_, center=c_)
        return float(g_lo @ lo + g_hi @ hi)

    h = 1e-5
    for vec, grad, which in ((x, gx, 0), (u, gu, 1), (rad, gr, 2), (c, gc, 3)):
        for i in range(len(vec)):
            e = np.zeros_like(vec)
            e[i] = h
            args_p = [x, u, rad, c]
            args_m = [x, u, rad, c]
            args_p[which] = vec + e
            args_m[which] = vec - e
            fd = (L(*args_p) - L(*args_m)) / (2 * h)
            assert fd == pytest.approx(grad[i], rel=2e-3, abs=2e-6), (which, i)
    # where the nominal lies outside the box, that side's end is the nominal: the centre and the radius move
    # only the other end, so their gradients there are equal (both d/d(far end)) and the centre's is not 0
    out = np.abs(c - a) > rad
    assert np.all(np.abs(gc[out]) > 0)
    far_sign = np.sign(c - a)[out]     # the far end is c + rho where c > a, c - rho where c < a
    assert np.allclose(gr[out], far_sign * gc[out], rtol=1e-9, atol=1e-12)


def test_oracle_gradient_zonotope_hull_matches_finite_differences():
    """The oracle's gradient for a zonotope set taken as its interval hull (Eq. 21), w.r.t. (x~, u~, G,
    centre), vs central differences of the box bound at radii sum_g |G_ig| (h = 1e-5, FP64); the centre
    sits off the nominal, inside the box in half the coordinates and outside in the other half. Two
    special cases: a diagonal G is the box of radii |G_ii| (the box gradient times sign(G_ii)), and a zero
    generator entry gets no gradient."""
    w = inputs.tanh_mlp(n_traj=1, N=2, widths=(10, 16, 16, 6))
    rng = np.random.default_rng(18)
    t = 1
    x, u = w.x_nom[t].astype(np.float64), w.u_nom[t].astype(np.float64)
    a = np.concatenate([x, u])
    n, p = a.size, 5
    G = rng.normal(size=(n, p)) * 0.02
    G[3, 2] = 0.0
    rad = np.abs(G).sum(axis=1)
    scale = np.where(np.arange(n) % 2 == 0, 0.5, 2.0) * rng.choice([-1.0, 1.0], n)
    c = a + scale * rad
    g_lo = rng.normal(size=6)
    g_hi = rng.normal(size=6)
    gx, gu, gG, gc = crown.zono_hull_remainder_vjp(w.Ws, w.bs, "tanh", x, u, G, g_lo, g_hi, center=c)

    def L(x_, u_, G_, c_):
        lo, hi, _ = crown.box_remainder(w.Ws, w.bs, "tanh", x_, u_, np.abs(G_).sum(axis=1), center=c_)
        return float(g_lo @ lo + g_hi @ hi)

    h = 1e-5
    for vec, grad, which in ((x, gx, 0), (u, gu, 1), (c, gc, 3)):
        for i in range(len(vec)):
            e = np.zeros_like(vec)
            e[i] = h
            args_p = [x, u, G, c]
            args_m = [x, u, G, c]
            args_p[which] = vec + e
            args_m[which] = vec - e
            fd = (L(*args_p) - L(*args_m)) / (2 * h)
            assert fd == pytest.approx(grad[i], rel=2e-3, abs=2e-6), (which, i)
    for (i, g) in ((0, 0), (1, 4), (5, 2), (n - 1, 3), (7, 1)):
        Gp, Gm = G.copy(), G.copy()
        Gp[i, g] += h
        Gm[i, g] -= h
        fd = (L(x, u, Gp, c) - L(x, u, Gm, c)) / (2 * h)
        assert fd == pytest.approx(gG[i, g], rel=2e-3, abs=2e-6), (i, g)
    assert gG[3, 2] == 0.0
    # the row of dL/dG is dL/d(half-width) times sign(G): one magnitude per row
    mag = np.abs(gG)
    nz = G != 0
    for i in range(n):
        assert np.allclose(mag[i][nz[i]], mag[i][nz[i]].max(), rtol=1e-12, atol=0)
    # a diagonal G is the box of radii |G_ii|
    d = rng.normal(size=n) * 0.03
    gx2, gu2, gG2 = crown.zono_hull_remainder_vjp(w.Ws, w.bs, "tanh", x, u, np.diag(d), g_lo, g_hi)
    bx, bu, br = crown.box_remainder_vjp(w.Ws, w.bs, "tanh", x, u, np.abs(d), g_lo, g_hi)
    assert np.allclose(gx2, bx, rtol=1e-12, atol=1e-14) and np.allclose(gu2, bu, rtol=1e-12, atol=1e-14)
    assert np.allclose(np.diag(gG2), br * np.sign(d), rtol=1e-12, atol=1e-14)
    assert np.all(gG2[~np.eye(n, dtype=bool)] == 0.0)


def test_proposer_gradients_and_adam_closed_form():
    rng = np.random.default_rng(16)
    Ws = [rng.normal(size=(7, 5)) * 0.4, rng.normal(size=(6, 7)) * 0.4, rng.normal(size=(4, 6)) * 0.4]
    bs = [rng.normal(size=7) * 0.1, rng.normal(size=6) * 0.1, rng.normal(size=4) * 0.1]
    X = rng.normal(size=(9, 5))
    Tg = rng.normal(size=(9, 4))
    loss, gWs, gbs = proposer.loss_and_grads((Ws, bs), X, Tg)
    for li in range(3):
        for (i, j) in ((0, 0), (1, 2), (3, 1)):
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[li][i, j] += 1e-6
            Wm[li][i, j] -= 1e-6
            fd = (proposer.loss_and_grads((Wp, bs), X, Tg)[0] - proposer.loss_and_grads((Wm, bs), X, Tg)[0]) / 2e-6
            assert fd == pytest.approx(gWs[li][i, j], rel=1e-5, abs=1e-9)
    # Adam's first step moves each parameter by lr * g / (|g| + eps): ~ lr * sign(g)
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -1e-3, 2.0])
    p1, m, v = proposer.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_proposer_bf16_rounding_matches_torch():
    """The oracle's BF16 operand rounding is round-to-nearest-even, as torch's bfloat16 cast."""
    rng = np.random.default_rng(17)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.005859375, -2.5, 3e38])]).astype(np.float32)
    ref = torch.as_tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(proposer.bf16(x), ref)
    # with rounding on, gradients still match finite differences of the rounded loss at a smooth point
    Ws = [rng.normal(size=(6, 4)) * 0.5, rng.normal(size=(5, 6)) * 0.5, rng.normal(size=(3, 5)) * 0.5]
    bs = [rng.normal(size=6) * 0.1, rng.normal(size=5) * 0.1, rng.normal(size=3) * 0.1]
    X = rng.normal(size=(7, 4))
    Tg = rng.normal(size=(7, 3))
    l0, g0, _ = proposer.loss_and_grads((Ws, bs), X, Tg)
    l1, g1, _ = proposer.loss_and_grads((Ws, bs), X, Tg, bf16_ops=True)
    assert abs(l1 - l0) < 5e-2 * abs(l0)
    for a, b in zip(g0, g1):
        assert np.max(np.abs(a - b)) < 5e-2 * np.abs(a).max()


def test_ibp_intermediate_single_hidden_layer_equals_crown():
    """With one hidden layer there is no intermediate layer to bound, so the IBP variant is CROWN itself."""
    Ws, bs = _net((5, 24, 3), 30)
    for act in ("relu", "tanh"):
        a = np.random.default_rng(31).normal(size=5)
        r = np.full(5, 0.2)
        c1 = crown.box_remainder(Ws, bs, act, a[:3], a[3:], r, residual=True)
        c2 = crown.box_remainder(Ws, bs, act, a[:3], a[3:], r, residual=True, intermediate="ibp")
        assert np.array_equal(c1[0], c2[0]) and np.array_equal(c1[1], c2[1])


def test_ibp_layer_is_exact_for_monotone_nets():
    """Positive diagonal first layer, non-negative second layer, monotone activation: every layer-2
    pre-activation is increasing in every input, so its range over a box is [z(lo), z(hi)], which IBP
    must reproduce."""
    rng = np.random.default_rng(32)
    W1 = np.diag(rng.uniform(0.5, 2.0, 4))
    b1 = rng.normal(size=4) * 0.1
    W2 = rng.uniform(0.0, 1.0, (5, 4))
    b2 = rng.normal(size=5) * 0.1
    t = lambda x: torch.tensor(x)
    for act in ("relu", "tanh"):
        lo, hi = rng.normal(size=4) - 0.5, None
        hi = lo + rng.uniform(0.1, 1.0, 4)
        l1, u1 = W1 @ lo + b1, W1 @ hi + b1
        l2, u2 = crown.ibp_layer(t(W2), t(b2), act, t(l1), t(u1))
        f = (lambda z: np.maximum(z, 0)) if act == "relu" else np.tanh
        assert np.allclose(l2.numpy(), W2 @ f(l1) + b2, rtol=1e-14, atol=1e-15)
        assert np.allclose(u2.numpy(), W2 @ f(u1) + b2, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("act", ["relu", "tanh"])
def test_ibp_intermediate_bounds_and_remainder_are_sound(act):
    """Sampled pre-activations of every hidden layer lie in the IBP bounds, and the resulting Thm. 3
    bound contains the sampled true remainder; ReLU: it contains the exact range by enumeration."""
    rng = np.random.default_rng(33)
    Ws, bs = _net((6, 16, 16, 16, 4), 34)
    Wt = [torch.tensor(W) for W in Ws]
    bt = [torch.tensor(b) for b in bs]
    a = rng.normal(size=6)
    lo, hi = a - 0.25, a + 0.25
    _, _, _, _, bounds = crown.crown(Wt, bt, act, torch.tensor(lo), torch.tensor(hi), intermediate="ibp")
    P = sampling.box_points(lo, hi, 20000, rng)
    h = torch.tensor(P)
    for i, (l, u) in enumerate(bounds):
        z = h @ Wt[i].T + bt[i]
        assert torch.all(z >= l - 1e-12) and torch.all(z <= u + 1e-12)
        h = crown.act_fn(act, z)
    r_lo, r_hi, J, _ = crown.remainder_bounds(Wt, bt, act, torch.tensor(a), torch.tensor(lo), torch.tensor(hi),
                                              residual=False, intermediate="ibp")
    R = sampling.remainders(sampling.mlp_f_batch(Ws, bs, act, residual=False), a, J.numpy(), P)
    assert np.all(R.min(0) >= r_lo.numpy() - 1e-12) and np.all(R.max(0) <= r_hi.numpy() + 1e-12)
    if act == "relu":
        el, eh, _ = exact.relu_exact_range(Ws, bs, a, lo, hi, residual=False)
        assert np.all(r_lo.numpy() <= el + 1e-12) and np.all(r_hi.numpy() >= eh - 1e-12)


def test_zonotope_crown_with_diagonal_generators_is_the_box_version():
    """G = diag(r) makes the zonotope the box c +- r: every concretisation ||Lambda G||_{1,r} = |Lambda| r,
    so the zonotope version reproduces the box version."""
    w = inputs.tanh_mlp(seed=4300, n_traj=1, N=3, widths=(12, 24, 24, 6))
    for t in range(w.T):
        G = np.diag(w.radii[t].astype(np.float64))
        zl, zh, zJ = crown.zono_remainder(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], G)
        bl, bh, bJ = crown.box_remainder(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t])
        assert np.allclose(zl, bl, rtol=1e-12, atol=1e-15) and np.allclose(zh, bh, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("act", ["relu", "tanh"])
def test_zonotope_crown_sound_on_sampled_zonotope_points(act):
    """Thm. 3 over a skewed zonotope (more generators than dimensions, centre off the nominal): every
    sampled point's true remainder lies in the bound, vertices of the generator cube included; and the
    hull construction contains the nominal."""
    rng = np.random.default_rng(35)
    Ws, bs = _net((6, 16, 16, 4), 36)
    n_x = 4
    a = rng.normal(size=6)
    G = rng.normal(size=(6, 9)) * 0.05
    c = a + rng.normal(size=6) * 0.02
    ch, Gh = crown.zono_hull_nominal(torch.tensor(a), torch.tensor(c), torch.tensor(G))
    xi = np.linalg.lstsq(Gh.numpy(), a - ch.numpy(), rcond=None)[0]
    assert np.allclose(Gh.numpy() @ xi + ch.numpy(), a)
    rl, rh, J = crown.zono_remainder(Ws, bs, act, a[:n_x], a[n_x:], G, center=c, residual=False)
    Xi = np.concatenate([rng.uniform(-1, 1, (20000, 9)), rng.choice([-1.0, 1.0], (5000, 9))])
    P = c + Xi @ G.T
    R = sampling.remainders(sampling.mlp_f_batch(Ws, bs, act, residual=False), a, J, P)
    assert np.all(R.min(0) >= rl - 1e-12) and np.all(R.max(0) <= rh + 1e-12)
    # the exact concretisation is never looser than the box hull's at the first layer
    W1 = torch.tensor(Ws[0])
    assert torch.all((W1 @ torch.tensor(G)).abs().sum(1) <= W1.abs() @ torch.tensor(np.abs(G).sum(1)) + 1e-15)
