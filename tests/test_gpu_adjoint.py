"""GPU adjoint of the CROWN bound against the oracle's gradient (itself pinned by central finite
differences in FP64, tests/test_oracle_crown.py), through the C ABI and the autograd.Function.

Tolerance: the kernels differentiate the same algorithm in FP32 (relaxation cases fixed at the evaluation
point). The relaxation points themselves are the FP32 bounds, which sit about 1e-3 (relative to the
interval widths; the forward's stated slack) away from the FP64 ones, and the slopes' derivatives move
with them, so the gradient agrees to that order relative to the gradient's scale:
    |g_gpu - g_oracle| <= 5e-3 max|g_oracle| + 5e-3 |g_oracle|
per timestep and input group (x~, u~, radii).
"""
import numpy as np
import pytest
import torch

from oracle import crown
from paper_2607_01203_b300 import binding, inputs
from paper_2607_01203_b300.autograd import leb_bounds

pytestmark = pytest.mark.gpu


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda().float()


def check(w, rows, seed=0, prec="fp32"):
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, prec)
    rng = np.random.default_rng(seed)
    g_lo = rng.normal(size=(len(rows), w.n_x)).astype(np.float32)
    g_hi = rng.normal(size=(len(rows), w.n_x)).astype(np.float32)
    x = _t(w.x_nom[rows]).requires_grad_(True)
    u = _t(w.u_nom[rows]).requires_grad_(True)
    r = _t(w.radii[rows]).requires_grad_(True)
    lo, hi = leb_bounds(h, x, u, r)
    (lo * _t(g_lo)).sum().backward(retain_graph=True)
    (hi * _t(g_hi)).sum().backward()
    gx, gu, gr = x.grad.cpu().numpy(), u.grad.cpu().numpy(), r.grad.cpu().numpy()
    for i, t in enumerate(rows):
        ox, ou, orr = crown.box_remainder_vjp(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], g_lo[i], g_hi[i],
                                              w.residual)
        for got, ref in ((gx[i], ox), (gu[i], ou), (gr[i], orr)):
            tol = 5e-3 * np.abs(ref).max() + 5e-3 * np.abs(ref)
            assert np.all(np.abs(got - ref) <= tol), (t, np.max(np.abs(got - ref) / (np.abs(ref).max() + 1e-30)))


@pytest.mark.parametrize("act", ["tanh", "relu"])
def test_small_nets(act):
    w = inputs.tanh_mlp(seed=4100, n_traj=1, N=4, widths=(10, 16, 16, 6)) if act == "tanh" else \
        inputs.relu_mlp(seed=4101, N=4, widths=(10, 16, 16, 6))
    check(w, list(range(w.T)))


def test_workload_subset():
    w = inputs.tanh_mlp(n_traj=1, N=50)
    check(w, [0, 7, 33])


def test_tensor_core_handle_uses_the_same_adjoint():
    w = inputs.tanh_mlp(seed=4102, n_traj=1, N=3, widths=(64, 128, 128, 32))
    check(w, [0, 1, 2], prec="fp16")
