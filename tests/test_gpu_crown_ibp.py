"""GPU parity of the IBP-intermediate variant of CROWN (hidden-layer bounds by interval bound
propagation, output by back-substitution and Thm. 3) against the FP64 oracle, through the C ABI.

Tolerance as for the CROWN paths: |gpu - oracle| <= 1e-5 w_l + 2 eps_l + 2^-20 s_l, eps_l the kernel's
stated slack (its inflation, the slack of its FP32 relaxation arithmetic, and the distance of its FP32
IBP bounds from the exact ones); soundness by sampling the true remainder."""
import numpy as np
import pytest
import torch

from oracle import crown, sampling
from paper_2607_01203_b300 import binding, inputs

pytestmark = pytest.mark.gpu


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to("cuda", torch.float32)


def run(w, prec, intermediate="ibp", rows=None):
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, prec, intermediate=intermediate)
    sel = slice(None) if rows is None else rows
    out = h.bounds(_t(w.x_nom[sel]), _t(w.u_nom[sel]), radii=_t(w.radii[sel]), want_eps=True)
    torch.cuda.synchronize()
    return h, {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


def parity(w, g, rows):
    for i, t in enumerate(rows):
        ol, oh, J = crown.box_remainder(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], w.residual,
                                        intermediate="ibp")
        eps = g["eps"][i].astype(np.float64)
        tol = 1e-5 * (oh - ol) + 2 * eps + 2.0 ** -20 * np.maximum(np.abs(ol), np.abs(oh))
        dl, dh = np.abs(g["r_lo"][i] - ol), np.abs(g["r_hi"][i] - oh)
        assert np.all(dl <= tol) and np.all(dh <= tol), (t, np.max(dl / tol), np.max(dh / tol))


@pytest.mark.parametrize("act,prec", [("tanh", "fp32"), ("relu", "fp32"), ("tanh", "fp16"), ("relu", "bf16")])
def test_small_nets_vs_oracle(act, prec):
    w = inputs.tanh_mlp(seed=3200, n_traj=1, N=8, widths=(64, 128, 128, 32)) if act == "tanh" else \
        inputs.relu_mlp(seed=3201, N=8, widths=(64, 128, 128, 32))
    _, g = run(w, prec)
    assert g["flags"][0] == 0
    parity(w, g, list(range(w.T)))


def test_tanh_workload_subset_and_soundness():
    """The 224-512-512-512-168 tanh net (FP16 tensor cores for the output chain): sampled timesteps
    against the oracle, and the sampled true remainder inside the bound."""
    w = inputs.tanh_mlp(n_traj=2, N=50)
    rows = [0, 1, 17, 49, 50, 99]
    h, g = run(w, "fp16", rows=rows)
    assert g["flags"][0] == 0
    parity(w, g, rows)
    f = sampling.mlp_f_batch(w.Ws, w.bs, w.act)
    rng = np.random.default_rng(12)
    for i, t in enumerate(rows[:3]):
        a = w.nominal()[t].astype(np.float64)
        lin = np.concatenate([g["A"][i], g["B"][i]], axis=1).astype(np.float64)
        R = sampling.remainders(f, a, lin, sampling.box_points(a - w.radii[t], a + w.radii[t], 100_000, rng))
        assert np.all(R >= g["r_lo"][i]) and np.all(R <= g["r_hi"][i])
    # the adjoint differentiates the CROWN variant only
    x, u, r = _t(w.x_nom[:2]), _t(w.u_nom[:2]), _t(w.radii[:2])
    with pytest.raises(binding.LebError):
        h.bounds_backward(x, u, r, torch.zeros(2, w.n_x, device="cuda"), torch.zeros(2, w.n_x, device="cuda"))
