"""GPU adjoint of the CROWN bound against the oracle's gradient (itself pinned by central finite
differences in FP64, tests/test_oracle_crown.py), through the C ABI and the autograd.Function.

Tolerance, per timestep, relative to the gradient's scale (the max over x~, u~ and radii together: the
x~, u~ parts are often 10-400 times smaller than the radii part, and every part moves by amounts set by
that scale):
    |g_gpu - g_oracle| <= rel max|g_oracle| + rel |g_oracle|.
The kernels differentiate the same algorithm with every relaxation case fixed at the evaluation point;
what differs is where the relaxation points sit. On the CUDA-core (FP32) path they are the FP32 bounds,
within the path's stated slack of the FP64 ones (0.4 % of the widths on the benchmark net, measured by
the benchmark's formats row), and the worst gradient error measured on B300 over these tests is 2.3e-4:
rel = 1e-3. The tensor-core adjoint also rounds its GEMM operands to the handle's format (unit roundoff
u = 2^-11 FP16, 2^-8 BF16), which moves the recomputed bounds and every chain product by a few u
relative; measured worst 1.1e-3 (2.3 u) for FP16 and 7.5e-3 (1.9 u) for BF16: rel = 1e-3 + 4 u.
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


def check(w, rows, seed=0, prec="fp32", rel=1e-3, report=False):
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
    worst = 0.0
    for i, t in enumerate(rows):
        ox, ou, orr = crown.box_remainder_vjp(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], g_lo[i], g_hi[i],
                                              w.residual)
        ref = np.concatenate([ox, ou, orr])
        got = np.concatenate([gx[i], gu[i], gr[i]])
        scale = np.abs(ref).max()          # the timestep's gradient scale (all of x~, u~, radii)
        err = np.max(np.abs(got - ref) / (scale + np.abs(ref) + 1e-30))
        worst = max(worst, err)
        if not report:
            tol = rel * scale + rel * np.abs(ref)
            assert np.all(np.abs(got - ref) <= tol), (t, np.max(np.abs(got - ref) / (scale + 1e-30)))
    print(f"adjoint {prec} {w.act} rows {len(rows)}: worst |err| / (max|g| + |g|) = {worst:.2e}")
    return worst


@pytest.mark.parametrize("act", ["tanh", "relu"])
def test_small_nets(act):
    w = inputs.tanh_mlp(seed=4100, n_traj=1, N=4, widths=(10, 16, 16, 6)) if act == "tanh" else \
        inputs.relu_mlp(seed=4101, N=4, widths=(10, 16, 16, 6))
    check(w, list(range(w.T)))


def test_workload_subset():
    w = inputs.tanh_mlp(n_traj=1, N=50)
    check(w, [0, 7, 33])


U_OP = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("act", ["tanh", "relu"])
def test_tensor_core_adjoint_small_nets(prec, act):
    w = inputs.tanh_mlp(seed=4102, n_traj=1, N=3, widths=(64, 128, 128, 32)) if act == "tanh" else \
        inputs.relu_mlp(seed=4103, N=3, widths=(64, 128, 128, 32))
    check(w, [0, 1, 2], prec=prec, rel=1e-3 + 4 * U_OP[prec])


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tensor_core_adjoint_workload_many_tiles_per_cta(prec):
    """100 timesteps of the full network: 400 output tiles and 800 tiles per hidden target, more than
    one per SM, so every CTA carries several tiles through the scratch and the barriers."""
    w = inputs.tanh_mlp(n_traj=2, N=50)
    check(w, [0, 7, 33, 60, 99], prec=prec, rel=1e-3 + 4 * U_OP[prec])


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tensor_core_adjoint_pairs_odd_item_count(prec):
    """The tensor-core adjoint runs on CTA pairs that take two tiles a pass: 301 timesteps of a net with
    one tile per timestep for every target (32 outputs: 96 of 126 rows; 64 hidden neurons: 128 rows) give
    an odd tile count, several passes per pair and a pair whose last pass has a tile past the end (it
    must write nothing). The gradient of the whole batch at sampled timesteps, the last included, against
    the oracle."""
    w = inputs.tanh_mlp(seed=4108, n_traj=1, N=301, widths=(64, 64, 64, 32))
    assert w.T == 301
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, prec)
    rng = np.random.default_rng(21)
    g_lo = rng.normal(size=(w.T, w.n_x)).astype(np.float32)
    g_hi = rng.normal(size=(w.T, w.n_x)).astype(np.float32)
    gx, gu, gr, fl = h.bounds_backward(_t(w.x_nom), _t(w.u_nom), _t(w.radii), _t(g_lo), _t(g_hi))
    torch.cuda.synchronize()
    assert int(fl.item()) == 0
    got_all = torch.cat([gx, gu, gr], 1).cpu().numpy()
    assert np.all(np.isfinite(got_all))
    rel = 1e-3 + 4 * U_OP[prec]
    for t in (0, 1, 147, 148, 149, 296, 299, 300):
        ox, ou, orr = crown.box_remainder_vjp(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], g_lo[t],
                                              g_hi[t], w.residual)
        ref = np.concatenate([ox, ou, orr])
        err = np.abs(got_all[t] - ref)
        scale_t = np.abs(ref).max()
        assert np.all(err <= rel * scale_t + rel * np.abs(ref)), (t, np.max(err / (scale_t + 1e-30)))


def test_tensor_core_adjoint_full_network_one_timestep():
    """One timestep of the full network: 4 output tiles and 8 tiles per hidden target, so the CTA pairs'
    grid shrinks to two or four CTAs and every pass has both of its tiles."""
    w = inputs.tanh_mlp(n_traj=1, N=1)
    assert w.T == 1
    check(w, [0], prec="fp16", rel=1e-3 + 4 * U_OP["fp16"])


def test_tensor_core_adjoint_uneven_widths():
    """Widths that leave partial M-tiles, a partial K-block of the inputs and a partial output tile (96
    inputs, 192 and 128 hidden, 40 outputs: 120 of the tile's 126 rows)."""
    w = inputs.tanh_mlp(seed=4104, n_traj=1, N=3, widths=(96, 192, 128, 40))
    check(w, [0, 1, 2], prec="fp16", rel=1e-3 + 4 * U_OP["fp16"])


def test_tensor_core_adjoint_matches_cuda_core_adjoint():
    """The tensor-core adjoint against the FP32 CUDA-core adjoint on a 256-timestep slice of the full
    workload (both differentiate the same algorithm; they differ by operand rounding and by the
    relaxation points, i.e. the bounds of each forward path)."""
    w = inputs.tanh_mlp(n_traj=8, N=32)
    rng = np.random.default_rng(5)
    g_lo = _t(rng.normal(size=(w.T, w.n_x)))
    g_hi = _t(rng.normal(size=(w.T, w.n_x)))
    x, u, r = _t(w.x_nom), _t(w.u_nom), _t(w.radii)
    outs = []
    for prec in ("fp32", "fp16"):
        h = binding.mlp(w.Ws, w.bs, w.act, w.residual, prec)
        gx, gu, gr, flags = h.bounds_backward(x, u, r, g_lo, g_hi)
        torch.cuda.synchronize()
        assert flags.item() == 0
        outs.append(torch.cat([gx, gu, gr], 1).cpu().numpy())
    ref, got = outs
    scale = np.abs(ref).max(axis=1, keepdims=True)
    err = np.abs(got - ref) / (scale + np.abs(ref))
    print(f"tensor-core vs CUDA-core adjoint: worst {err.max():.2e}, mean {err.mean():.2e}")
    assert err.max() <= 1e-2 and err.mean() <= 1e-3


def test_adjoint_from_saved_forward_state():
    """leb_bounds_backward_saved right after leb_bounds on the same inputs (FP32 handle): the forward left
    exactly the bounds the adjoint differentiates, so the gradient equals the recomputing adjoint (up to
    the order of its atomic sums) and matches the FP64 oracle; reduced-precision handles refuse."""
    w = inputs.tanh_mlp(n_traj=2, N=50)
    rows = [0, 7, 33, 60, 99]
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, "fp32")
    rng = np.random.default_rng(6)
    g_lo = rng.normal(size=(len(rows), w.n_x)).astype(np.float32)
    g_hi = rng.normal(size=(len(rows), w.n_x)).astype(np.float32)
    x, u, r = _t(w.x_nom[rows]), _t(w.u_nom[rows]), _t(w.radii[rows])
    recompute = torch.cat(h.bounds_backward(x, u, r, _t(g_lo), _t(g_hi))[:3], 1).cpu().numpy()
    h.bounds(x, u, radii=r)
    gx, gu, gr, fl = h.bounds_backward(x, u, r, _t(g_lo), _t(g_hi), saved=True)
    torch.cuda.synchronize()
    assert int(fl.item()) == 0
    got = torch.cat([gx, gu, gr], 1).cpu().numpy()
    for i, t in enumerate(rows):
        ref = np.concatenate(crown.box_remainder_vjp(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], g_lo[i],
                                                     g_hi[i], w.residual))
        assert np.all(np.abs(got[i] - ref) <= 1e-3 * (np.abs(ref).max() + np.abs(ref))), t
    d = np.abs(got - recompute) / (np.abs(recompute).max(axis=1, keepdims=True) + np.abs(recompute))
    assert d.max() <= 1e-5
    h16 = binding.mlp(w.Ws, w.bs, w.act, w.residual, "fp16")
    h16.bounds(x, u, radii=r)
    with pytest.raises(binding.LebError):
        h16.bounds_backward(x, u, r, _t(g_lo), _t(g_hi), saved=True)


def test_adjoint_takes_a_batch_of_ragged_trajectories():
    """leb_bounds_backward with a leb_batch of trajectories of uneven horizon gives the gradient of the
    same timesteps in a row (every timestep's bound is independent); a batch of uneven chain lengths is
    refused, and so is a malformed one."""
    w = inputs.tanh_mlp(seed=4105, n_traj=1, N=9, widths=(64, 128, 128, 32))
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, "fp16")
    rng = np.random.default_rng(8)
    g_lo, g_hi = _t(rng.normal(size=(w.T, w.n_x))), _t(rng.normal(size=(w.T, w.n_x)))
    x, u, r = _t(w.x_nom), _t(w.u_nom), _t(w.radii)
    plain = torch.cat(h.bounds_backward(x, u, r, g_lo, g_hi)[:3], 1)
    offs = torch.tensor([0, 2, 7, 9], dtype=torch.int32, device="cuda")
    gx, gu, gr, fl = h.bounds_backward(x, u, r, g_lo, g_hi, traj_offsets=offs)
    torch.cuda.synchronize()
    assert int(fl.item()) == 0
    got = torch.cat([gx, gu, gr], 1)
    scale = plain.abs().max(dim=1, keepdim=True).values + plain.abs()
    assert torch.all((got - plain).abs() <= 1e-5 * scale)   # the adjoint's atomic sums, up to their order
    lib = binding.lib()
    bd = binding.BatchDesc(3, offs.data_ptr(), offs.data_ptr())
    sd = h.set_desc(radii=r)
    ws = h.workspace(w.T)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    args = (w.T, x.data_ptr(), u.data_ptr(), binding.C.byref(sd), g_lo.data_ptr(), g_hi.data_ptr(), gx.data_ptr(),
            gu.data_ptr(), gr.data_ptr(), ws.data_ptr(), ws.numel(), flags.data_ptr(), None)
    assert lib.leb_bounds_backward(h.h, binding.C.byref(bd), *args) == binding.LEB_ERR_UNSUPPORTED
    bad = binding.BatchDesc(0, offs.data_ptr(), None)
    assert lib.leb_bounds_backward(h.h, binding.C.byref(bad), *args) == binding.LEB_ERR_INVALID_ARG


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_off_centre_box_gradient(prec):
    """leb_bounds_backward_box for boxes centred off the nominal (hulled with it): dL/d(x~, u~, radii,
    centre) against the FP64 oracle's gradient (itself pinned by central differences). Half the
    coordinates have the nominal inside the box, half outside it (that side's end is then the nominal).
    Tolerance as for centred sets, rel = 1e-3 on FP32 handles; the reduced formats' operand rounding moves
    these gradients further than the centred ones (measured worst 1.3e-3 = 2.6 u FP16, 1.6e-2 = 4.0 u BF16;
    FP32 4.0e-5), so rel = 1e-3 + 6 u there. The centred call is unchanged: leb_bounds_backward refuses a
    centre (no place for its gradient), and quad-chain handles take centred sets only."""
    w = inputs.tanh_mlp(seed=4106, n_traj=1, N=4, widths=(64, 128, 128, 32))
    rng = np.random.default_rng(9)
    a = w.nominal().astype(np.float64)
    scale = np.where(rng.uniform(size=a.shape) < 0.5, 0.5, 2.0) * rng.choice([-1.0, 1.0], a.shape)
    c = (a + scale * w.radii).astype(np.float32)
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, prec)
    g_lo = rng.normal(size=(w.T, w.n_x)).astype(np.float32)
    g_hi = rng.normal(size=(w.T, w.n_x)).astype(np.float32)
    x, u, r, cc = _t(w.x_nom), _t(w.u_nom), _t(w.radii), _t(c)
    gx, gu, gr, gc, fl = h.bounds_backward(x, u, r, _t(g_lo), _t(g_hi), center=cc)
    torch.cuda.synchronize()
    assert int(fl.item()) == 0
    got_all = torch.cat([gx, gu, gr, gc], 1).cpu().numpy()
    rel = 1e-3 if prec == "fp32" else 1e-3 + 6 * U_OP[prec]
    worst = 0.0
    for t in range(w.T):
        ox, ou, orr, oc = crown.box_remainder_vjp(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], w.radii[t], g_lo[t],
                                                  g_hi[t], w.residual, center=c[t].astype(np.float64))
        ref = np.concatenate([ox, ou, orr, oc])
        got = got_all[t]
        scale_t = np.abs(ref).max()
        err = np.abs(got - ref)
        worst = max(worst, float(np.max(err / (scale_t + np.abs(ref)))))
        assert np.all(err <= rel * scale_t + rel * np.abs(ref)), (t, np.max(err / (scale_t + 1e-30)))
    print(f"off-centre adjoint {prec}: worst |err| / (max|g| + |g|) = {worst:.2e}")
    # the API's contract
    lib = binding.lib()
    sd = h.set_desc(radii=r, center=cc)
    ws = h.workspace(w.T)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    args = (w.T, x.data_ptr(), u.data_ptr(), binding.C.byref(sd), _t(g_lo).data_ptr(), _t(g_hi).data_ptr(),
            gx.data_ptr(), gu.data_ptr(), gr.data_ptr())
    assert lib.leb_bounds_backward(h.h, None, *args, ws.data_ptr(), ws.numel(), flags.data_ptr(), None) == \
        binding.LEB_ERR_INVALID_ARG
    q = inputs.planar_quad()
    hq = binding.quad_chain(1, **q.params)
    with pytest.raises(binding.LebError):
        hq.bounds_backward(_t(q.x_nom), _t(q.u_nom), _t(q.radii), _t(np.ones((q.T, q.n_x))), _t(np.ones((q.T, q.n_x))),
                           center=_t(np.concatenate([q.x_nom, q.u_nom], 1)))


@pytest.mark.parametrize("prec,n_gen,centred", [("fp32", 5, True), ("fp32", 37, False), ("fp16", 37, True),
                                                ("fp16", 5, False), ("bf16", 37, False)])
def test_zonotope_hull_gradient(prec, n_gen, centred):
    """leb_bounds_backward_zono: the adjoint of the bound over a zonotope set's interval hull (Eq. 21),
    dL/d(x~, u~, G[, centre]) against the FP64 oracle's gradient (pinned by central differences). G's
    row l1 norms are the box workload's radii (so the hull is that box), 5 or 37 generators (a warp's
    lanes and a ragged second pass), one entry per row set to 0; off-centre sets put the nominal inside
    the hull in half the coordinates, outside in the rest. Tolerances as for box sets: dL/dG_ig is the
    half-width gradient times sign(G_ig)."""
    w = inputs.tanh_mlp(seed=4107, n_traj=1, N=4, widths=(64, 128, 128, 32))
    rng = np.random.default_rng(10 + n_gen)
    a = w.nominal().astype(np.float64)
    share = rng.uniform(0.1, 1.0, size=(w.T, w.n, n_gen))
    share[:, :, n_gen // 2] = 0.0
    share /= share.sum(axis=2, keepdims=True)
    G = (w.radii[:, :, None] * share * rng.choice([-1.0, 1.0], share.shape)).astype(np.float32)
    rad = np.abs(G.astype(np.float64)).sum(axis=2)
    c = None
    if not centred:
        scale = np.where(rng.uniform(size=a.shape) < 0.5, 0.5, 2.0) * rng.choice([-1.0, 1.0], a.shape)
        c = (a + scale * rad).astype(np.float32)
    h = binding.mlp(w.Ws, w.bs, w.act, w.residual, prec)
    g_lo = rng.normal(size=(w.T, w.n_x)).astype(np.float32)
    g_hi = rng.normal(size=(w.T, w.n_x)).astype(np.float32)
    x, u = _t(w.x_nom), _t(w.u_nom)
    gx, gu, gG, gc, fl = h.bounds_backward_zono(x, u, _t(G), _t(g_lo), _t(g_hi), center=None if c is None else _t(c))
    torch.cuda.synchronize()
    assert int(fl.item()) == 0
    assert (gc is None) == centred
    gG = gG.cpu().numpy()
    assert np.all(gG[:, :, n_gen // 2] == 0.0)
    parts = [gx, gu, torch.as_tensor(gG.reshape(w.T, -1))] + ([] if c is None else [gc])
    got_all = torch.cat([p.cpu() for p in parts], 1).numpy()
    rel = 1e-3 if prec == "fp32" else 1e-3 + 6 * U_OP[prec]
    worst = 0.0
    for t in range(w.T):
        out = crown.zono_hull_remainder_vjp(w.Ws, w.bs, w.act, w.x_nom[t], w.u_nom[t], G[t].astype(np.float64),
                                            g_lo[t], g_hi[t], w.residual,
                                            center=None if c is None else c[t].astype(np.float64))
        ref = np.concatenate([out[0], out[1], out[2].reshape(-1)] + ([] if c is None else [out[3]]))
        got = got_all[t]
        scale_t = np.abs(ref).max()
        err = np.abs(got - ref)
        worst = max(worst, float(np.max(err / (scale_t + np.abs(ref)))))
        assert np.all(err <= rel * scale_t + rel * np.abs(ref)), (t, np.max(err / (scale_t + 1e-30)))
    print(f"zonotope-hull adjoint {prec} n_gen={n_gen} centred={centred}: worst = {worst:.2e}")
    # the API's contract: the box entry points refuse a zonotope, the zonotope one a box; quad chains none
    lib = binding.lib()
    sd = h.set_desc(G=_t(G))
    ws = h.workspace(w.T)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    gr = torch.empty(w.T, w.n, device="cuda")
    args = (w.T, x.data_ptr(), u.data_ptr(), binding.C.byref(sd), _t(g_lo).data_ptr(), _t(g_hi).data_ptr(),
            gx.data_ptr(), gu.data_ptr(), gr.data_ptr())
    assert lib.leb_bounds_backward(h.h, None, *args, ws.data_ptr(), ws.numel(), flags.data_ptr(), None) == \
        binding.LEB_ERR_UNSUPPORTED
    assert lib.leb_bounds_backward_box(h.h, None, *args, None, ws.data_ptr(), ws.numel(), flags.data_ptr(),
                                       None) == binding.LEB_ERR_UNSUPPORTED
    sb = h.set_desc(radii=_t(w.radii))
    args_b = (w.T, x.data_ptr(), u.data_ptr(), binding.C.byref(sb), _t(g_lo).data_ptr(), _t(g_hi).data_ptr(),
              gx.data_ptr(), gu.data_ptr(), gr.data_ptr())
    assert lib.leb_bounds_backward_zono(h.h, None, *args_b, None, ws.data_ptr(), ws.numel(), flags.data_ptr(),
                                        None) == binding.LEB_ERR_INVALID_ARG
    q = inputs.planar_quad()
    hq = binding.quad_chain(1, **q.params)
    with pytest.raises(binding.LebError):
        hq.bounds_backward_zono(_t(q.x_nom), _t(q.u_nom), _t(np.full((q.T, q.n, 2), 0.01)),
                                _t(np.ones((q.T, q.n_x))), _t(np.ones((q.T, q.n_x))))
