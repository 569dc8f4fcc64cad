"""Pins of the a-priori rounding analysis of reduced-precision back-substitution (oracle/tc_rounding.py)
against actual rounded arithmetic and against the plain FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import crown, tc_rounding as tr
from paper_2607_01203_b300 import inputs

F64 = torch.float64


def _operands(seed, R, K, N):
    g = torch.Generator().manual_seed(seed)
    a = torch.randn(R, K, generator=g, dtype=F64)
    # magnitudes over many decades, some in FP16's subnormal range, some exact zeros
    a = a * torch.pow(10.0, torch.randint(-9, 2, (R, K), generator=g).to(F64))
    a[:, ::17] = 0.0
    W = torch.randn(K, N, generator=g, dtype=F64) / K ** 0.5
    return a, W


@pytest.mark.parametrize("fmt", ["fp16", "bf16", "fp32"])
@pytest.mark.parametrize("K", [64, 512])
def test_stage_bound_covers_emulated_rounded_stage(fmt, K):
    """The bound holds entrywise on a stage computed with rounded operands and FP32 sums, and is not
    vacuous (the actual error reaches a visible fraction of it)."""
    a, W = _operands(100 + K, 64, K, 96)
    err = (tr.emulate_stage(a, W, fmt) - a @ W).abs()
    bound = tr.stage_error_bound(a, W, fmt)
    assert torch.all(err <= bound)
    # the worst-case FP32 accumulation term (K u) dominates the FP32 bound, while rounding errors of a
    # random sum grow like sqrt(K) u / 2; the reduced formats' operand rounding is reached closely
    assert float((err / bound).max()) > (1e-3 if fmt == "fp32" else 0.05)


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_stage_bound_terms_are_needed(fmt):
    """Planted mistakes on constructed worst cases: an operand and a weight each 0.49 ulp above 1 both
    round down to 1, so the rounded product misses the exact one by ~2 u_op, which the bound without its
    weight-rounding term |W - W~| does not cover; an operand 0.49 ulp above 1 times an exact weight misses
    by ~u_op, which the bound without the operand-rounding term does not cover. The full bound covers both."""
    ulp = 2.0 * tr.unit_roundoff(fmt)
    x = 1.0 + 0.49 * ulp
    for a, W, dropped in ((x, x, "weight"), (x, 1.0, "operand")):
        a_t = torch.tensor([[a]], dtype=F64)
        W_t = torch.tensor([[W]], dtype=F64)
        err = (tr.emulate_stage(a_t, W_t, fmt) - a_t @ W_t).abs()
        assert torch.all(err <= tr.stage_error_bound(a_t, W_t, fmt))
        Wt = tr.round_to(W_t, fmt)
        g = tr.gamma(1)
        if dropped == "weight":
            wrong = a_t.abs() @ ((tr.unit_roundoff(fmt) + 2.0 ** -24 + g) * Wt.abs())
        else:
            wrong = a_t.abs() @ ((2.0 ** -24 + g) * Wt.abs() + (W_t - Wt).abs())
        assert torch.all(err > wrong), dropped


def test_envelope_with_k0_is_the_oracle():
    """With the inflation applied zero times the envelope is Thm. 3 of the plain oracle."""
    w = inputs.tanh_mlp(seed=3100, n_traj=1, N=4, widths=(64, 128, 128, 32))
    for t in range(w.T):
        ol, oh, _ = crown.box_remainder(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], w.residual)
        el, eh, il, iu = tr.remainder_envelope(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], "fp16", 0.0)
        s = np.maximum(np.abs(ol), np.abs(oh))
        assert np.allclose(el, ol, rtol=0, atol=1e-12 * s.max()) and np.allclose(eh, oh, rtol=0, atol=1e-12 * s.max())
        assert np.all(il > 0) and np.all(iu > 0)


def test_envelope_nesting_and_format_scaling():
    """k = 2 contains k = 1 contains the oracle; the inflation scales with the format's unit roundoff
    (BF16's is 8 times FP16's); FP32's, dominated by the accumulation term gamma_K, is far below both."""
    w = inputs.tanh_mlp(seed=3101, n_traj=1, N=3, widths=(64, 128, 128, 32))
    for t in range(w.T):
        args = (w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t])
        ol, oh, _ = crown.box_remainder(*args, w.residual)
        e1l, e1h, il16, iu16 = tr.remainder_envelope(*args, "fp16", 1.0)
        e2l, e2h, _, _ = tr.remainder_envelope(*args, "fp16", 2.0)
        _, _, il8, iu8 = tr.remainder_envelope(*args, "bf16", 1.0)
        _, _, il32, _ = tr.remainder_envelope(*args, "fp32", 1.0)
        assert np.all(e2l <= e1l) and np.all(e1l <= ol) and np.all(e2h >= e1h) and np.all(e1h >= oh)
        ratio = il8 / il16
        assert np.all((ratio > 4) & (ratio < 12)), ratio
        assert np.all(il32 < 0.1 * il16)


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_jacobian_error_bound_covers_emulated_chain(fmt):
    """The a-priori Jacobian-chain bound holds elementwise on chains computed with rounded operands, also on
    the adversarial cancelling net (whose Jacobian is small next to its terms), and is not vacuous."""
    nets = [inputs.tanh_mlp(seed=3102, n_traj=1, N=2, widths=(64, 512, 512, 32)), inputs.tanh_mlp_cancelling(N=2)]
    worst = 0.0
    for w in nets:
        for t in range(w.T):
            a = w.nominal()[t].astype(np.float64)
            J = crown.jacobian([crown.to_t(W) for W in w.Ws], [crown.to_t(b) for b in w.bs], w.act,
                               crown.to_t(a)).numpy()
            err = np.abs(tr.emulate_jacobian(w.Ws, w.bs, w.act, a, fmt) - J)
            bound = tr.jacobian_error_bound(w.Ws, w.bs, w.act, a, fmt)
            assert np.all(err <= bound)
            worst = max(worst, float(np.max(err / bound)))
    assert worst > 1e-3   # a worst-case bound: random rounding errors average out over the sums


# ---- zonotope stage (sets concretised exactly with a reduced-precision last product) ------------------
def _zono_operands(seed, R, n, p, offset):
    g = torch.Generator().manual_seed(seed)
    M = torch.randn(R, n, generator=g, dtype=F64)
    M = M * torch.pow(10.0, torch.randint(-9, 2, (R, n), generator=g).to(F64))
    M[:, ::13] = 0.0
    a = torch.randn(n, generator=g, dtype=F64).to(torch.float32).to(F64)
    G = 0.05 * torch.randn(n, p, generator=g, dtype=F64)
    c = (a + offset * torch.randn(n, generator=g, dtype=F64)).to(torch.float32).to(F64)
    return M, a, G, c


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
@pytest.mark.parametrize("offset", [0.0, 0.02])
def test_zono_stage_allowance_covers_emulation(fmt, offset):
    """min over the zonotope of M Delta computed with rounded operands, FP32 sums and an FP32 cd stays
    within the allowance of the exact FP64 value, row by row, and the allowance is not vacuous."""
    M, a, G, c = _zono_operands(200 + int(100 * offset), 48, 224, 30, offset)
    cd = 0.5 * (c - a)
    h = 2 * cd.abs() + G.abs().sum(dim=1)
    err = (tr.emulate_zono_stage(M, c, a, G, fmt) - tr.zono_min(M, cd, G)).abs()
    allow = tr.zono_stage_allowance(M, h, G.shape[1], fmt)
    assert torch.all(err <= allow)
    assert float((err / allow).max()) > 0.05


def test_zono_min_is_the_vertex_minimum():
    """The closed form M cd - |M cd| - sum_g |M G_g| is the minimum of M Delta over the zonotope's vertices
    (brute force over all 2^(p+1) sign patterns of a small one)."""
    M, a, G, c = _zono_operands(210, 5, 6, 7, 0.3)
    cd = 0.5 * (c - a)
    Bfull = torch.cat([-cd[:, None], G], dim=1)      # Delta = cd + [-cd | G] xi
    signs = torch.tensor(np.array(np.meshgrid(*[[-1.0, 1.0]] * 8)).reshape(8, -1), dtype=F64)
    vals = M @ (cd[:, None] + Bfull @ signs)
    assert torch.allclose(vals.min(dim=1).values, tr.zono_min(M, cd, G), rtol=0, atol=1e-12)


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_zono_stage_terms_are_needed(fmt):
    """Constructed worst case: every M_i and every generator entry 0.49 ulp above a representable value,
    all positive, so both round down and every |v_g| comes out ~2 u_op too small; V, the minimum, comes out
    too large by ~2 u_op sum_i h_i (the unsafe direction). The allowance covers it to within a few percent;
    without the generator-rounding u (or the operand-rounding u) in cz it does not."""
    u = tr.unit_roundoff(fmt)
    x = 1.0 + 0.49 * 2.0 * u
    n, p = 64, 8
    M = torch.full((1, n), x, dtype=F64)
    G = torch.full((n, p), x * 0.25, dtype=F64)
    a = torch.zeros(n, dtype=F64)
    err = tr.emulate_zono_stage(M, a, a, G, fmt) - tr.zono_min(M, torch.zeros(n, dtype=F64), G)
    h = G.abs().sum(dim=1)
    allow = tr.zono_stage_allowance(M, h, p, fmt)
    assert torch.all(err > 0) and torch.all(err <= allow)
    assert float((err / allow).min()) > 0.9
    cz, wadd, zc1, zc2, _ = tr.zono_stage_constants(n, p, fmt)
    g = tr.gamma(64)
    for cz_wrong in ((g * (1 + u) + u) * (1 + u) + 2.0 ** -23, g * (1 + u) ** 2 + u + 2.0 ** -23):
        wrong = M.abs() @ (cz_wrong * h + wadd) + zc1 * float(h.sum()) + zc2
        assert torch.all(err > wrong)


def test_zono_envelope_with_k0_is_the_oracle_and_nests():
    """With the inflation applied zero times the zonotope envelope is the plain oracle's Thm. 3 over the
    zonotope; k = 2 contains k = 1 contains it; a zonotope with one generator per input of the box's
    radii reproduces the box envelope's output (same set, hull = box)."""
    w = inputs.tanh_mlp(seed=3103, n_traj=1, N=3, widths=(64, 128, 128, 32))
    rng = np.random.default_rng(3)
    for t in range(w.T):
        G = rng.normal(size=(w.n, 9)) * 0.02
        c = w.nominal()[t] + 0.01 * rng.normal(size=w.n)
        args = (w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], G, c)
        ol, oh, _ = crown.zono_remainder(*args[:5], G, center=c, residual=w.residual)
        e0l, e0h, il, iu = tr.zono_remainder_envelope(*args, "fp16", 0.0)
        e1l, e1h, _, _ = tr.zono_remainder_envelope(*args, "fp16", 1.0)
        e2l, e2h, _, _ = tr.zono_remainder_envelope(*args, "fp16", 2.0)
        s = max(np.abs(ol).max(), np.abs(oh).max())
        assert np.allclose(e0l, ol, rtol=0, atol=1e-12 * s) and np.allclose(e0h, oh, rtol=0, atol=1e-12 * s)
        assert np.all(e2l <= e1l) and np.all(e1l <= ol) and np.all(e2h >= e1h) and np.all(e1h >= oh)
        assert np.all(il > 0) and np.all(iu > 0)
    t = 0
    D = np.diag(w.radii[t].astype(np.float64))
    zl, zh, _, _ = tr.zono_remainder_envelope(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], D, None, "fp16", 0.0)
    bl, bh, _, _ = tr.remainder_envelope(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], "fp16", 0.0)
    assert np.allclose(zl, bl, rtol=0, atol=1e-10) and np.allclose(zh, bh, rtol=0, atol=1e-10)
