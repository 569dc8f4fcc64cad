"""GPU parity of the tensor-core CROWN chain (FP16 or BF16 operands, FP32 accumulation in TMEM) against
the FP64 oracle, through the C ABI, with a rounding allowance the test computes itself.

The tensor-core path evaluates the oracle's algorithm (Thms. 2-3) with rounded GEMM operands and moves
every bound outward by a rigorous a-priori inflation. The test does not take that inflation from the
kernel: ``oracle/tc_rounding.py`` computes it in FP64 on the oracle's own Lambda chains from the
operand format's unit roundoff, the FP16/BF16 rounding of the weights and gamma_K (the standard
dot-product error bound), pinned on CPU against emulated rounded stages. Per bound the test asserts
  * one-sided containment of the FP64 oracle: gpu_lo <= oracle_lo + tol, gpu_hi >= oracle_hi - tol,
    tol = 1e-5 w + 2^-20 s (w the oracle's width, s its magnitude);
  * no wider than the worst case the analysis allows: inside the envelope with every back-substituted
    bound widened by twice its inflation (once for the actual rounding error, once for the inflation
    the kernel subtracts), up to the same tol;
  * the kernel's stated slack eps (2 x its inflation) within a small factor of twice the test's figure
    (measured on B300: 1.0007-1.0063 across the workloads, FP16 and BF16), so an over- or under-stated
    inflation fails.
Soundness is checked separately by sampling the true remainder w.r.t. the returned A, B, including an
adversarial net on which the bound without its inflation is violated.
"""
import numpy as np
import pytest
import torch

from oracle import crown, sampling, tc_rounding as tr
from paper_2607_01203_b300 import binding, inputs

pytestmark = pytest.mark.gpu

EPS_FACTOR = (0.98, 1.10)   # kernel eps / (2 x the test's inflation)


def _t(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to("cuda", dtype)


def run(w, prec, rows=None):
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, prec)
    sel = slice(None) if rows is None else rows
    out = h.bounds(_t(w.x_nom[sel]), _t(w.u_nom[sel]), radii=_t(w.radii[sel]), want_eps=True)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


def parity(w, g, rows, fmt, idx=None):
    """The three assertions above for every row of every listed timestep; returns the mean width ratio
    gpu / oracle and the extreme eps ratios."""
    wr, er = [], []
    for i, t in enumerate(rows):
        ii = i if idx is None else idx[i]
        args = (w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t])
        ol, oh, J = crown.box_remainder(*args, w.residual)
        e2l, e2h, _, _ = tr.remainder_envelope(*args, fmt, 2.0)
        _, _, il, iu = tr.remainder_envelope(*args, fmt, 1.0)   # the inflation as the kernel applies it
        gl, gh = g["r_lo"][ii].astype(np.float64), g["r_hi"][ii].astype(np.float64)
        tol = 1e-5 * (oh - ol) + 2.0 ** -20 * np.maximum(np.abs(ol), np.abs(oh))
        assert np.all(gl <= ol + tol) and np.all(gh >= oh - tol), (t, np.max(gl - ol - tol), np.max(oh - gh - tol))
        assert np.all(gl >= e2l - tol) and np.all(gh <= e2h + tol), (t, np.max(e2l - gl - tol), np.max(gh - e2h - tol))
        ratio = g["eps"][ii].astype(np.float64) / (2.0 * np.maximum(il, iu))
        assert np.all((ratio >= EPS_FACTOR[0]) & (ratio <= EPS_FACTOR[1])), (t, ratio.min(), ratio.max())
        er += [ratio.min(), ratio.max()]
        wr.append(np.mean((gh - gl) / (oh - ol)))
        # the returned [A B] against the FP64 Jacobian: the a-priori bound of the rounded Jacobian chain
        # (oracle/tc_rounding.py) plus 1e-5 of the absolute chain for the kernel's FP32 slopes sigma'(z^)
        AB = np.concatenate([g["A"][ii], g["B"][ii]], axis=1)
        a = w.nominal()[t].astype(np.float64)
        jb = tr.jacobian_error_bound(w.Ws, w.bs, w.act, a, fmt)
        jb_scale = jb / (1.01 * tr.unit_roundoff(fmt))
        assert np.all(np.abs(AB - J) <= jb + 1e-5 * jb_scale + 2.0 ** -23 * np.abs(J)), np.max(np.abs(AB - J) / jb)
    return float(np.mean(wr)), float(min(er)), float(max(er))


def small_net(act="tanh", seed=3100):
    return inputs.tanh_mlp(seed=seed, n_traj=1, N=8, widths=(64, 128, 32)) if act == "tanh" else \
        inputs.relu_mlp(seed=seed, N=8, widths=(64, 128, 128, 32))


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
@pytest.mark.parametrize("act", ["tanh", "relu"])
def test_small_nets_tc_vs_oracle(act, fmt):
    w = small_net(act)
    g = run(w, fmt)
    assert g["flags"][0] == 0
    parity(w, g, list(range(w.T)), fmt)


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_tc_full_size_sampled_parity(fmt):
    """The 128 x 50 tanh-MLP batch of the benchmark (224-512-512-512-168) in its launch configuration;
    64 sampled timesteps and the last one against the oracle and the test's own inflation figure."""
    w = inputs.tanh_mlp()
    g = run(w, fmt)
    assert g["flags"][0] == 0
    rng = np.random.default_rng(12)
    rows = sorted(rng.choice(w.T - 1, 64, replace=False).tolist()) + [w.T - 1]
    sub = {k: (v[rows] if isinstance(v, np.ndarray) and v.ndim >= 2 else v) for k, v in g.items()}
    wratio, emin, emax = parity(w, sub, rows, fmt)
    print(f"{fmt}: width gpu / oracle {wratio:.3f}, eps / test figure in [{emin:.4f}, {emax:.4f}]")


def test_tc_soundness_sampled():
    w = inputs.tanh_mlp(n_traj=1, N=4)
    for fmt in ("fp16", "bf16"):
        g = run(w, fmt)
        f = sampling.mlp_f_batch(w.Ws, w.bs, w.act)
        rng = np.random.default_rng(11)
        for t in range(w.T):
            a = w.nominal()[t].astype(np.float64)
            lin = np.concatenate([g["A"][t], g["B"][t]], axis=1).astype(np.float64)
            P = sampling.box_points(a - w.radii[t], a + w.radii[t], 200_000, rng)
            R = sampling.remainders(f, a, lin, P)
            assert np.all(R >= g["r_lo"][t]) and np.all(R <= g["r_hi"][t])


def test_adversarial_net_needs_the_inflation():
    """Large weights and cancelling pairs of hidden neurons (inputs.tanh_mlp_cancelling, box radius 1e-3):
    the Jacobian the kernel returns carries operand-rounding errors that are large next to the curvature
    part of the remainder. Sampled remainders (box points plus, per row, the two vertices at which the
    error of the returned linearization, (J - A) delta, is extreme) stay inside the bounds in both
    formats; with BF16 operands the same bounds without their rounding inflation (moved inward by eps / 2,
    the inflation the kernel states it subtracted) are violated."""
    w = inputs.tanh_mlp_cancelling(radius=1e-3)
    f = sampling.mlp_f_batch(w.Ws, w.bs, w.act)
    rng = np.random.default_rng(21)
    deflated_violations = {}
    for fmt in ("fp16", "bf16"):
        g = run(w, fmt)
        assert g["flags"][0] == 0
        parity(w, g, list(range(w.T)), fmt)
        n_defl = 0
        for t in range(w.T):
            a = w.nominal()[t].astype(np.float64)
            rho = w.radii[t].astype(np.float64)
            lin = np.concatenate([g["A"][t], g["B"][t]], axis=1).astype(np.float64)
            _, _, J = crown.box_remainder(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], w.residual)
            D = np.sign(J - lin)
            P = np.concatenate([a + D * rho, a - D * rho, sampling.box_points(a - rho, a + rho, 6000, rng)])
            R = sampling.remainders(f, a, lin, P)
            gl, gh = g["r_lo"][t].astype(np.float64), g["r_hi"][t].astype(np.float64)
            assert np.all(R >= gl) and np.all(R <= gh), (fmt, t)
            e = g["eps"][t].astype(np.float64) / 2.0
            n_defl += int(np.sum((R > gh - e) | (R < gl + e)))
        deflated_violations[fmt] = n_defl
    print("sampled violations of the bounds without their inflation:", deflated_violations)
    assert deflated_violations["bf16"] > 0


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_tc_plans_bit_identical_and_autotune(fmt):
    """The tensor-core chain plans (job widths 256 and 128: how the final stage's and narrow hidden stages'
    columns are grouped into MMA jobs) give the same bits, forward (bounds, A, B, stated slack) and adjoint,
    on the benchmark's net (final stage 224 columns: a partial second job) and on a net of uneven widths
    (hidden stages of 192 and 128 columns); leb_autotune times them and keeps one, with the same bits. (The
    adjoint's atomic sums are compared up to their order.)"""
    nets = [inputs.tanh_mlp(n_traj=4, N=50), inputs.tanh_mlp(seed=4104, n_traj=1, N=6, widths=(96, 192, 128, 40))]
    for w in nets:
        h = binding.mlp(w.Ws, w.bs, w.act, w.residual, fmt)
        assert h.plan_count() == 2
        x, u, r = _t(w.x_nom), _t(w.u_nom), _t(w.radii)
        rng = np.random.default_rng(31)
        glo, ghi = _t(rng.normal(size=(w.T, w.n_x))), _t(rng.normal(size=(w.T, w.n_x)))
        ref = None
        for p in range(2):
            h.select_plan(p)
            assert f"tc_job_cols={(256, 128)[p]}" in h.plan()
            o = h.bounds(x, u, radii=r, want_eps=True)
            gx, gu, gr, fl = h.bounds_backward(x, u, r, glo, ghi)
            torch.cuda.synchronize()
            assert int(o["flags"].item()) == 0 and int(fl.item()) == 0
            got = [o["r_lo"].clone(), o["r_hi"].clone(), o["A"].clone(), o["B"].clone(), o["eps"].clone(),
                   torch.cat([gx, gu, gr], 1)]
            if ref is None:
                ref = got
            else:
                for a_, b_ in zip(ref[:5], got[:5]):
                    assert torch.equal(a_, b_), p
                # the adjoint sums its per-neuron terms with atomic adds, whose order varies from run to run
                # (also within one plan): equal up to that reordering
                g0, g1 = ref[5].double(), got[5].double()
                scale = g0.abs().max(dim=1, keepdim=True).values + g0.abs()
                assert torch.all((g0 - g1).abs() <= 1e-5 * scale), p
        h.select_plan(-1)
        h.autotune(w.T, binding.SET_BOX)
        assert "autotune=measured" in h.plan()
        o = h.bounds(x, u, radii=r, want_eps=True)
        torch.cuda.synchronize()
        assert torch.equal(o["r_lo"], ref[0]) and torch.equal(o["r_hi"], ref[1])
        print(fmt, w.Ws[0].shape, h.plan())
