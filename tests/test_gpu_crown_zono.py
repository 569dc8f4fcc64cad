"""GPU parity of CROWN concretised exactly over zonotope tube sets (LEB_SET_ZONO_EXACT, FP32 CUDA-core
chains) against the FP64 oracle, through the C ABI.

Tolerance as for the FP32 CROWN path: |gpu - oracle| <= 1e-5 w_l + 2 eps_l + 2^-20 s_l, plus the rounding
of the zonotope sums (each |sum_m Lambda_m G_mg| carries gamma_n sum |Lambda_m| |G_mg|, which the kernel
adds): 2 gamma_n sum_g sum_m |M_m| |G_mg| <= 2 gamma_n ||M||_1 ||G||_max n_gen, taken with the oracle's M."""
import numpy as np
import pytest
import torch

from oracle import crown, sampling
from paper_2607_01203_b300 import binding, inputs

pytestmark = pytest.mark.gpu


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to("cuda", torch.float32)


def _zono_workload(act, seed, T=6, n_gen=12, widths=(10, 32, 32, 6), offset=0.0):
    w = inputs.relu_mlp(seed=seed, N=T, widths=widths) if act == "relu" else \
        inputs.tanh_mlp(seed=seed, n_traj=1, N=T, widths=widths)
    rng = np.random.default_rng(seed)
    G = (rng.normal(size=(w.T, w.n, n_gen)) * 0.03).astype(np.float32)
    c = (w.nominal() + offset * rng.normal(size=(w.T, w.n))).astype(np.float32)
    return w, G, c


@pytest.mark.parametrize("act,offset", [("tanh", 0.0), ("relu", 0.0), ("tanh", 0.02), ("relu", 0.02)])
def test_zonotope_exact_parity_and_soundness(act, offset):
    w, G, c = _zono_workload(act, 4400 + int(offset * 100), offset=offset)
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, "fp32")
    center = _t(c) if offset else None
    out = h.bounds(_t(w.x_nom), _t(w.u_nom), G=_t(G), center=center, want_eps=True, zono_exact=True)
    hull = h.bounds(_t(w.x_nom), _t(w.u_nom), G=_t(G), center=center)
    torch.cuda.synchronize()
    assert int(out["flags"].item()) == 0
    g = {k: v.cpu().numpy() for k, v in out.items() if torch.is_tensor(v)}
    gh = {k: v.cpu().numpy() for k, v in hull.items() if torch.is_tensor(v)}
    n_gen = G.shape[2]
    gam = 1.01 * w.n * 2.0 ** -24
    f = sampling.mlp_f_batch(w.Ws, w.bs, w.act)
    rng = np.random.default_rng(5)
    narrower = 0
    for t in range(w.T):
        ol, oh, J = crown.zono_remainder(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], G[t].astype(np.float64),
                                         center=None if center is None else c[t].astype(np.float64))
        eps = g["eps"][t].astype(np.float64)
        zs = 2 * gam * n_gen * np.abs(G[t]).max() * (np.abs(J).sum(1) + 2.0)
        tol = 1e-5 * (oh - ol) + 2 * eps + 2.0 ** -20 * np.maximum(np.abs(ol), np.abs(oh)) + zs
        assert np.all(np.abs(g["r_lo"][t] - ol) <= tol) and np.all(np.abs(g["r_hi"][t] - oh) <= tol), t
        # soundness: sampled points of the zonotope (and of the segment to the nominal when off-centre)
        a = w.nominal()[t].astype(np.float64)
        Xi = np.concatenate([rng.uniform(-1, 1, (20000, n_gen)), rng.choice([-1.0, 1.0], (5000, n_gen))])
        P = c[t].astype(np.float64) + Xi @ G[t].astype(np.float64).T
        lin = np.concatenate([g["A"][t], g["B"][t]], axis=1).astype(np.float64)
        R = sampling.remainders(f, a, lin, P)
        assert np.all(R >= g["r_lo"][t]) and np.all(R <= g["r_hi"][t])
        narrower += np.sum(g["r_hi"][t] - g["r_lo"][t]) <= np.sum(gh["r_hi"][t] - gh["r_lo"][t])
    assert narrower >= w.T - 1   # the exact concretisation is (almost always) tighter than the hull's


def test_zonotope_exact_refused_where_not_built():
    w, G, _ = _zono_workload("tanh", 4500, widths=(64, 128, 128, 32))
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, "fp16")   # tensor-core chains: hull only
    with pytest.raises(binding.LebError):
        h.bounds(_t(w.x_nom), _t(w.u_nom), G=_t(G), zono_exact=True)
    q = inputs.planar_quad()
    hq = binding.quad_chain(1, **q.params)
    with pytest.raises(binding.LebError):
        hq.bounds(_t(q.x_nom), _t(q.u_nom), G=_t(np.zeros((q.T, 8, 2), np.float32)), zono_exact=True)
