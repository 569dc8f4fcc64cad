"""GPU parity of CROWN concretised exactly over zonotope tube sets (LEB_SET_ZONO_EXACT) against the FP64
oracle, through the C ABI: the FP32 CUDA-core chains and the tensor-core chains (FP16 / BF16 operands).

FP32 chains: tolerance as for the FP32 CROWN path, |gpu - oracle| <= 1e-5 w_l + 2 eps_l + 2^-20 s_l, plus
the rounding of the zonotope sums (each |sum_m Lambda_m G_mg| carries gamma_n sum |Lambda_m| |G_mg|, which
the kernel adds): 2 gamma_n sum_g sum_m |M_m| |G_mg| <= 2 gamma_n ||M||_1 ||G||_max n_gen, taken with the
oracle's M. Tensor-core chains: see the section below."""
import numpy as np
import pytest
import torch

from oracle import crown, sampling, tc_rounding as tr
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
    """Quad-chain handles take no exact zonotope; tensor-core MLP handles take at most 510 generators (the
    zonotope stage's 512 columns)."""
    w, G, _ = _zono_workload("tanh", 4500, widths=(64, 128, 128, 32), n_gen=511)
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, "fp16")
    with pytest.raises(binding.LebError):
        h.bounds(_t(w.x_nom), _t(w.u_nom), G=_t(G), zono_exact=True)
    q = inputs.planar_quad()
    hq = binding.quad_chain(1, **q.params)
    with pytest.raises(binding.LebError):
        hq.bounds(_t(q.x_nom), _t(q.u_nom), G=_t(np.zeros((q.T, 8, 2), np.float32)), zono_exact=True)


# ---- tensor-core chains (FP16 / BF16 operands) -------------------------------------------------------
# Same three assertions as the box sets' tensor-core test, with the test's own inflation model of
# oracle/tc_rounding.py (zono_remainder_envelope: the chain inflation of every stage plus the allowance of
# the zonotope stage, the extra product M [cd | G | -cd] with rounded operands, for every hidden layer and
# the output): one-sided containment of the FP64 oracle, inside the k = 2 envelope, and the kernel's
# stated slack within EPS_FACTOR of twice the model's inflation. The returned A, B are those of the box
# path (the Jacobian chain does not depend on the set).
EPS_FACTOR = (0.98, 1.10)


def tc_zono_parity(w, G, c, g, rows, fmt, idx=None):
    wr, er = [], []
    for i, t in enumerate(rows):
        ii = i if idx is None else idx[i]
        ct = None if c is None else c[t].astype(np.float64)
        Gt = G[t].astype(np.float64)
        ol, oh, _ = crown.zono_remainder(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], Gt, center=ct,
                                         residual=w.residual)
        args = (w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], Gt, ct)
        e2l, e2h, _, _ = tr.zono_remainder_envelope(*args, fmt, 2.0)
        _, _, il, iu = tr.zono_remainder_envelope(*args, fmt, 1.0)
        gl, gh = g["r_lo"][ii].astype(np.float64), g["r_hi"][ii].astype(np.float64)
        tol = 1e-5 * (oh - ol) + 2.0 ** -20 * np.maximum(np.abs(ol), np.abs(oh))
        assert np.all(gl <= ol + tol) and np.all(gh >= oh - tol), (t, np.max(gl - ol - tol), np.max(oh - gh - tol))
        assert np.all(gl >= e2l - tol) and np.all(gh <= e2h + tol), (t, np.max(e2l - gl - tol), np.max(gh - e2h - tol))
        ratio = g["eps"][ii].astype(np.float64) / (2.0 * np.maximum(il, iu))
        assert np.all((ratio >= EPS_FACTOR[0]) & (ratio <= EPS_FACTOR[1])), (t, ratio.min(), ratio.max())
        er += [ratio.min(), ratio.max()]
        wr.append(np.mean((gh - gl) / (oh - ol)))
    return float(np.mean(wr)), float(min(er)), float(max(er))


def _tc_run(w, G, c, fmt):
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, fmt)
    center = None if c is None else _t(c)
    z = h.bounds(_t(w.x_nom), _t(w.u_nom), G=_t(G), center=center, want_eps=True, zono_exact=True)
    hull = h.bounds(_t(w.x_nom), _t(w.u_nom), G=_t(G), center=center)
    torch.cuda.synchronize()
    assert int(z["flags"].item()) == 0 and int(hull["flags"].item()) == 0
    assert torch.equal(z["A"], hull["A"]) and torch.equal(z["B"], hull["B"])
    g = {k: v.cpu().numpy() for k, v in z.items() if torch.is_tensor(v)}
    gh = {k: v.cpu().numpy() for k, v in hull.items() if torch.is_tensor(v)}
    return g, gh


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
@pytest.mark.parametrize("act,offset", [("tanh", 0.0), ("relu", 0.0), ("tanh", 0.02), ("relu", 0.02)])
def test_tc_zonotope_parity_and_soundness(act, offset, fmt):
    w, G, c = _zono_workload(act, 4600 + int(offset * 100), widths=(64, 128, 128, 32), offset=offset)
    c = c if offset else None
    g, gh = _tc_run(w, G, c, fmt)
    wr, emin, emax = tc_zono_parity(w, G, c, g, list(range(w.T)), fmt)
    f = sampling.mlp_f_batch(w.Ws, w.bs, w.act)
    rng = np.random.default_rng(7)
    narrower = 0
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        cen = a if c is None else c[t].astype(np.float64)
        Xi = np.concatenate([rng.uniform(-1, 1, (20000, G.shape[2])), rng.choice([-1.0, 1.0], (5000, G.shape[2]))])
        P = cen + Xi @ G[t].astype(np.float64).T
        lin = np.concatenate([g["A"][t], g["B"][t]], axis=1).astype(np.float64)
        R = sampling.remainders(f, a, lin, P)
        assert np.all(R >= g["r_lo"][t]) and np.all(R <= g["r_hi"][t])
        narrower += np.sum(g["r_hi"][t] - g["r_lo"][t]) <= np.sum(gh["r_hi"][t] - gh["r_lo"][t])
    assert narrower >= w.T - 1
    print(f"{fmt} {act} offset {offset}: width / oracle {wr:.3f}, eps / model in [{emin:.4f}, {emax:.4f}]")


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_tc_zonotope_shapes(fmt):
    """Inputs not a multiple of 64 (96: a half-empty operand block of the zonotope stage), 300 generators
    (302 columns: two zonotope jobs, the second partial), uneven hidden widths, an off-centre set."""
    w, G, c = _zono_workload("tanh", 4700, T=4, n_gen=300, widths=(96, 192, 128, 40), offset=0.01)
    g, _ = _tc_run(w, G, c, fmt)
    tc_zono_parity(w, G, c, g, list(range(w.T)), fmt)


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_tc_zonotope_full_size_sampled(fmt):
    """The benchmark's tanh MLP (224-512-512-512-168) on 256 timesteps of a zonotope tube with 64
    generators, centred off the nominal, in the launch configuration of a full batch; 12 sampled
    timesteps against the oracle and the model."""
    w = inputs.tanh_mlp(n_traj=8, N=32)
    rng = np.random.default_rng(4800)
    G = (rng.normal(size=(w.T, w.n, 64)) * 0.3 * w.radii[:, :, None] / 8.0).astype(np.float32)
    c = (w.nominal() + 0.2 * w.radii * rng.uniform(-1, 1, size=(w.T, w.n))).astype(np.float32)
    g, gh = _tc_run(w, G, c, fmt)
    rows = sorted(rng.choice(w.T - 1, 11, replace=False).tolist()) + [w.T - 1]
    sub = {k: (v[rows] if isinstance(v, np.ndarray) and v.ndim >= 2 else v) for k, v in g.items()}
    wr, emin, emax = tc_zono_parity(w, G, c, sub, rows, fmt)
    gain = float(np.mean((g["r_hi"] - g["r_lo"]) / (gh["r_hi"] - gh["r_lo"])))
    print(f"{fmt} full size: width / oracle {wr:.3f}, eps / model in [{emin:.4f}, {emax:.4f}], "
          f"exact / hull width {gain:.3f}")
