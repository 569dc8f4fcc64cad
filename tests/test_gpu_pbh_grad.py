"""GPU parity of the adjoint of the PBH bound (Thm. 1; differentiable LEBs, Sec. IV-D) and of the nominal
refinement by projected gradient descent (Sec. VI-A, Table II), through the C ABI.

Tolerance of the gradient: the kernel differentiates the same algorithm as the FP64 oracle, with the
same interval selections, in FP32 (round to nearest, sincosf accurate to a few ulps at the rollouts'
angles of up to tens of radians), each entry a product of at most five factors; so per timestep
    |g - g_oracle| <= 1e-4 (max |g_oracle| + |g_oracle|),
and the entries the bound does not depend on are exactly zero.
"""
import numpy as np
import pytest
import torch

from oracle import dynamics, pbh, pbh_grad
from paper_2607_01203_b300 import binding, inputs

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()


def _workloads():
    yield inputs.planar_quad(), list(range(20))
    w = inputs.proposer_data(n_rollouts=4, N=50)          # 28-quadrotor chain, box sets
    yield w, [0, 1, 17, 49, 50, 99, 123, 150, 199]


def _handle(w):
    return binding.quad_chain(w.n_quads, **w.params, spring_k=w.spring_k)


@pytest.mark.parametrize("which", [0, 1])
def test_gradient_parity_with_oracle(which):
    w, rows = list(_workloads())[which]
    h = _handle(w)
    dyn = dynamics.QuadChain(w.n_quads, **w.params, spring_k=w.spring_k)
    rng = np.random.default_rng(40 + which)
    g_lo = rng.normal(size=(w.T, w.n_x)).astype(np.float32)
    g_hi = rng.normal(size=(w.T, w.n_x)).astype(np.float32)
    gx, gu, gr, fl = h.bounds_backward(_t(w.x_nom), _t(w.u_nom), _t(w.radii), _t(g_lo), _t(g_hi))
    torch.cuda.synchronize()
    assert int(fl.item()) == 0
    G = torch.cat([gx, gu, gr], 1).cpu().numpy().astype(np.float64)
    for t in rows:
        rx, ru, rr = pbh_grad.pbh_vjp(dyn, w.nominal()[t].astype(np.float64), w.radii[t].astype(np.float64),
                                     g_lo[t].astype(np.float64), g_hi[t].astype(np.float64))
        ref = np.concatenate([rx, ru, rr])
        tol = 1e-4 * (np.abs(ref).max() + np.abs(ref))
        assert np.all(np.abs(G[t] - ref) <= tol), (t, np.max(np.abs(G[t] - ref) / tol))
        assert np.all(G[t][ref == 0.0] == 0.0)


def test_gradient_full_batch_sampled():
    """The 28-quadrotor chain in the bench's size class (256 x 50 timesteps) in one launch, sampled
    timesteps against the oracle one by one."""
    w = inputs.proposer_data(n_rollouts=256, N=50)
    h = _handle(w)
    dyn = dynamics.QuadChain(w.n_quads, **w.params, spring_k=w.spring_k)
    g_lo = -np.ones((w.T, w.n_x), np.float32)
    g_hi = np.ones((w.T, w.n_x), np.float32)
    gx, gu, gr, fl = h.bounds_backward(_t(w.x_nom), _t(w.u_nom), _t(w.radii), _t(g_lo), _t(g_hi))
    torch.cuda.synchronize()
    assert int(fl.item()) == 0
    G = torch.cat([gx, gu, gr], 1).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(41)
    for t in sorted(rng.choice(w.T, 8, replace=False).tolist()) + [w.T - 1]:
        ref = np.concatenate(pbh_grad.pbh_vjp(dyn, w.nominal()[t].astype(np.float64), w.radii[t].astype(np.float64),
                                              g_lo[t], g_hi[t]))
        assert np.all(np.abs(G[t] - ref) <= 1e-4 * (np.abs(ref).max() + np.abs(ref)))


@pytest.mark.parametrize("which", [0, 1])
def test_pgd_refinement(which):
    """Table II's comparison: projected gradient descent on the PBH width against random sampling of
    nominal points in the same box with as many bound evaluations (one forward and one backward per
    step, plus the final forward, against that many sampled forwards). The returned point lies in the
    box, its certified width is what leb_bounds gives there, it is never worse than the start, and PGD
    ends below the best sample on at least 90 % of the timesteps."""
    w, _ = list(_workloads())[which]
    if which == 1:
        w = inputs.subset(w, np.arange(64))
    h = _handle(w)
    eps, steps = 0.05, 10
    x0, u0, r = _t(w.x_nom), _t(w.u_nom), _t(w.radii)
    x1, u1, w0, w1, fl = h.refine_nominal_pgd(x0, u0, r, eps=eps, lr=eps / 5, steps=steps)
    torch.cuda.synchronize()
    assert int(fl.item()) == 0
    # inside the box; a float32 step may overshoot it by one rounding
    assert torch.all((x1 - x0).abs() <= eps * (1 + 1e-6) + 1e-6) and torch.all((u1 - u0).abs() <= eps * (1 + 1e-6) + 1e-6)
    o0 = h.bounds(x0, u0, radii=r, want_AB=False)
    o1 = h.bounds(x1, u1, radii=r, want_AB=False)
    torch.cuda.synchronize()
    wd0 = (o0["r_hi"] - o0["r_lo"]).sum(1)
    wd1 = (o1["r_hi"] - o1["r_lo"]).sum(1)
    assert torch.allclose(w0, wd0, rtol=1e-5) and torch.allclose(w1, wd1, rtol=1e-5)
    assert torch.all(w1 <= w0)
    # the FP64 oracle agrees on the refined point (the GPU width carries its outward rounding)
    dyn = dynamics.QuadChain(w.n_quads, **w.params, spring_k=w.spring_k)
    a1 = torch.cat([x1, u1], 1).cpu().numpy().astype(np.float64)
    for t in range(0, w.T, max(1, w.T // 8)):
        lo, hi = pbh.box_from_set(a1[t], radii=w.radii[t].astype(np.float64))
        ol, oh = pbh.pbh(dyn, a1[t], lo, hi)
        assert abs((oh - ol).sum() - float(w1[t])) <= 1e-4 * float(w1[t]) + 1e-6
    # random sampling with the same number of bound evaluations
    K = 2 * steps + 1
    g = torch.Generator(device="cuda").manual_seed(7)
    xs = (x0[:, None, :] + eps * (2 * torch.rand(w.T, K, w.n_x, device="cuda", generator=g) - 1)).reshape(-1, w.n_x)
    us = (u0[:, None, :] + eps * (2 * torch.rand(w.T, K, w.n_u, device="cuda", generator=g) - 1)).reshape(-1, w.n_u)
    rs = r[:, None, :].expand(w.T, K, w.n).reshape(-1, w.n).contiguous()
    os_ = h.bounds(xs.contiguous(), us.contiguous(), radii=rs, want_AB=False)
    torch.cuda.synchronize()
    ws = (os_["r_hi"] - os_["r_lo"]).sum(1).view(w.T, K).min(1).values
    better = (w1 < ws).float().mean().item()
    assert better >= 0.9, better
    assert float((w0 - w1).sum()) > 0
