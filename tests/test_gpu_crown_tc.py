"""GPU parity of the tensor-core CROWN chain (FP16 operands, FP32 accumulation in TMEM) against the
FP64 oracle, through the C ABI.

The tensor-core path evaluates the same algorithm as the oracle with rounded GEMM operands; it adds to
every bound a rigorous rounding inflation and states, per bound, eps_l = 2 x inflation + the slack of its
FP32 relaxation arithmetic. The tolerance is the one the FP32 path uses with that eps:
    |gpu - oracle| <= 1e-5 w_l + 2 eps_l + 2^-20 s_l.
Soundness is checked separately by sampling the true remainder w.r.t. the returned A, B.
"""
import numpy as np
import pytest
import torch

from oracle import crown, sampling
from paper_2607_01203_b300 import binding, inputs

pytestmark = pytest.mark.gpu


def _t(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to("cuda", dtype)


def run(w, prec, rows=None):
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, prec)
    sel = slice(None) if rows is None else rows
    out = h.bounds(_t(w.x_nom[sel]), _t(w.u_nom[sel]), radii=_t(w.radii[sel]), want_eps=True)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


def parity(w, g, rows, ab_tol):
    for i, t in enumerate(rows):
        ol, oh, J = crown.box_remainder(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], w.residual)
        eps = g["eps"][i].astype(np.float64)
        tol = 1e-5 * (oh - ol) + 2 * eps + 2.0 ** -20 * np.maximum(np.abs(ol), np.abs(oh))
        dl, dh = np.abs(g["r_lo"][i] - ol), np.abs(g["r_hi"][i] - oh)
        assert np.all(dl <= tol) and np.all(dh <= tol), (t, np.max(dl / tol), np.max(dh / tol))
        AB = np.concatenate([g["A"][i], g["B"][i]], axis=1)
        assert np.all(np.abs(AB - J) <= ab_tol * (np.abs(J).max() + 1e-30)), np.max(np.abs(AB - J))


def small_net(act="tanh", seed=3100):
    return inputs.tanh_mlp(seed=seed, n_traj=1, N=8, widths=(64, 128, 32)) if act == "tanh" else \
        inputs.relu_mlp(seed=seed, N=8, widths=(64, 128, 128, 32))


@pytest.mark.parametrize("act", ["tanh", "relu"])
def test_small_nets_tc_vs_oracle(act):
    w = small_net(act)
    g = run(w, "fp16")
    assert g["flags"][0] == 0
    parity(w, g, list(range(w.T)), ab_tol=2e-3)


def test_tanh_workload_subset_tc_vs_oracle():
    w = inputs.tanh_mlp(n_traj=2, N=50)
    rows = [0, 1, 17, 49, 50, 99]
    g = run(w, "fp16", rows)
    assert g["flags"][0] == 0
    parity(w, g, rows, ab_tol=2e-3)


def test_tc_soundness_sampled():
    w = inputs.tanh_mlp(n_traj=1, N=4)
    g = run(w, "fp16")
    f = sampling.mlp_f_batch(w.Ws, w.bs, w.act)
    rng = np.random.default_rng(11)
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lin = np.concatenate([g["A"][t], g["B"][t]], axis=1).astype(np.float64)
        P = sampling.box_points(a - w.radii[t], a + w.radii[t], 200_000, rng)
        R = sampling.remainders(f, a, lin, P)
        assert np.all(R >= g["r_lo"][t]) and np.all(R <= g["r_hi"][t])


def test_tc_full_size_sampled_parity():
    """The 128 x 50 tanh-MLP batch of the benchmark, in its launch configuration (FP16 tensor cores);
    sampled timesteps against the oracle one by one."""
    w = inputs.tanh_mlp()
    g = run(w, "fp16")
    assert g["flags"][0] == 0
    rng = np.random.default_rng(12)
    rows = sorted(rng.choice(w.T, 10, replace=False).tolist()) + [w.T - 1]
    sub = {k: (v[rows] if isinstance(v, np.ndarray) and v.ndim >= 2 else v) for k, v in g.items()}
    parity(w, sub, rows, ab_tol=2e-3)
