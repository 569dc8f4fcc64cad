"""GPU parity of the path-based Hessian bound (Thm. 1) against the FP64 oracle, through the C ABI.

Tolerance (derived from the FP32 arithmetic of the kernel): the GPU interval is an outward-rounded
enclosure of the same Eq. 15 evaluated on an outward-rounded hull, plus the term (J - A) Delta for the
FP32 Jacobian it returns. So, per row l,
  * containment: gpu_lo <= oracle_lo + 1e-12 s_l and gpu_hi >= oracle_hi - 1e-12 s_l (soundness w.r.t.
    the exact bound; s_l is the row's scale), and
  * width: gpu_w <= oracle_w (1 + 1e-5) + eps_l, with eps_l = 2^-18 sum_terms |H| |D_j| |D_k|
    + 2^-21 sum_j |J_lj| |D_j| (FP32 rounding of the terms and of the returned Jacobian entries)
    + 2 sum_terms |H| ((D_j + d_j)(D_k + d_k) - D_j D_k) with d_j = 2^-22 (|alpha~_j| + D_j), the
    widening from storing the box ends c -+ r as outward-rounded FP32 numbers.
"""
import math

import numpy as np
import pytest
import torch

from oracle import dynamics, pbh, sampling
from paper_2607_01203_b300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _t(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV, dtype)


def run_gpu(w, G=None, radii=None, center=None, batch=False, want_AB=True, handle=None, **kw):
    h = handle or binding.quad_chain(w.n_quads, **w.params, spring_k=w.spring_k)
    offs = _t(w.traj_offsets, torch.int32) if batch else None
    out = h.bounds(_t(w.x_nom), _t(w.u_nom), radii=None if radii is None else _t(radii),
                   G=None if G is None else _t(G), center=None if center is None else _t(center),
                   traj_offsets=offs, want_AB=want_AB, **kw)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


def tolerance(dyn, a, lo, hi, J):
    D = np.maximum(np.abs(lo - a), np.abs(hi - a))
    eps = 2.0 ** -21 * (np.abs(J) @ D)
    # coefficient magnitude of each Hessian entry (its trig factor replaced by 1, which covers the
    # absolute slack of the kernel's sin/cos enclosures)
    wide_lo, wide_hi = lo.copy(), hi.copy()
    for i in range(dyn.nq):
        wide_lo[dyn.ix(i, 2)], wide_hi[dyn.ix(i, 2)] = -4.0, 4.0
    # the kernel's box ends c -+ r are FP32 numbers rounded outward, so each half-width may grow by
    # about two ulps of |alpha~_j| + D_j
    dD = 2.0 ** -22 * (np.abs(a) + D)
    for row in range(dyn.n_x):
        for j, k, fn in dyn.hessian_terms(row):
            Hm = max(abs(v) for v in fn(wide_lo, wide_hi))
            eps[row] += 2.0 ** -18 * Hm * D[j] * D[k]
            eps[row] += 2.0 * Hm * ((D[j] + dD[j]) * (D[k] + dD[k]) - D[j] * D[k])
    return eps + 1e-30


def check_parity(dyn, a, lo, hi, gl, gh, A=None, B=None):
    ol, oh = pbh.pbh(dyn, a, lo, hi)
    J = dyn.jacobian(a)
    eps = tolerance(dyn, a, lo, hi, J)
    scale = np.abs(ol) + np.abs(oh) + 1e-300
    assert np.all(gl <= ol + 1e-12 * scale), np.max(gl - ol)
    assert np.all(gh >= oh - 1e-12 * scale), np.max(oh - gh)
    assert np.all((gh - gl) <= (oh - ol) * (1 + 1e-5) + eps), np.max((gh - gl) - (oh - ol) - eps)
    if A is not None:
        AB = np.concatenate([A, B], axis=1)
        assert np.all(np.abs(AB - J) <= 4 * 2.0 ** -23 * np.abs(J) + 1e-30)
    return ol, oh


def test_point_enclosures_contain_fp64_values():
    lib = binding.lib()
    rng = np.random.default_rng(0)
    xs = [rng.uniform(-10, 10, 200000), rng.uniform(-1e4, 1e4, 50000), rng.normal(size=50000) * 1e-3,
          np.array([0.0, -0.0, 1e-40, -1e-40, 3e38, -3e38, 1e-7, 8.0, 9.5, 20.0])]
    k = np.arange(-400, 400)
    for off in (0.0, 0.5):
        base = (k + off) * math.pi
        xs.append(np.concatenate([base, np.nextafter(base.astype(np.float32), np.float32(np.inf)),
                                  np.nextafter(base.astype(np.float32), np.float32(-np.inf))]))
    x = np.concatenate(xs).astype(np.float32)
    xt = _t(x)
    out = [torch.empty(x.size, 2, device=DEV) for _ in range(3)]
    binding.check(lib.leb_selftest_point_enclosures(xt.data_ptr(), x.size, out[0].data_ptr(), out[1].data_ptr(),
                                                    out[2].data_ptr(), None), "selftest")
    torch.cuda.synchronize()
    xd = x.astype(np.float64)
    for enc, ref in zip(out, (np.sin(xd), np.cos(xd), np.tanh(xd))):
        e = enc.cpu().numpy().astype(np.float64)
        assert np.all(e[:, 0] <= ref) and np.all(e[:, 1] >= ref)
        assert np.max(e[:, 1] - e[:, 0]) <= 2.0 ** -20


def test_planar_quad_parity_all_timesteps():
    w = inputs.planar_quad()
    dyn = dynamics.QuadChain(1, **w.params)
    g = run_gpu(w, radii=w.radii)
    assert g["flags"][0] == 0
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        check_parity(dyn, a, lo, hi, g["r_lo"][t], g["r_hi"][t], g["A"][t], g["B"][t])


def test_planar_quad_soundness_1e6_samples_per_set():
    """Zero violations of the true remainder (w.r.t. the returned FP32 A, B) over 10^6 points per set."""
    w = inputs.planar_quad()
    dyn = dynamics.QuadChain(1, **w.params)
    g = run_gpu(w, radii=w.radii)
    rng = np.random.default_rng(1)
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        lin = np.concatenate([g["A"][t], g["B"][t]], axis=1).astype(np.float64)
        for _ in range(4):
            P = sampling.box_points(lo, hi, 250000, rng)
            R = sampling.remainders(dyn.f_batch, a, lin, P)
            assert np.all(R >= g["r_lo"][t].astype(np.float64) - 1e-15)
            assert np.all(R <= g["r_hi"][t].astype(np.float64) + 1e-15)


def test_chain_zonotope_parity_small_ragged():
    """Several trajectories of uneven horizon, zonotope sets: every row of every timestep."""
    w = inputs.quad_chain(n_traj=5, horizon=(2, 7), n_quads=28)
    dyn = dynamics.QuadChain(28, **w.params, spring_k=w.spring_k)
    g = run_gpu(w, G=w.G, batch=True)
    plain = run_gpu(w, G=w.G, batch=False)
    assert np.array_equal(g["r_lo"], plain["r_lo"]) and np.array_equal(g["A"], plain["A"])
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, G=w.G[t])
        check_parity(dyn, a, lo, hi, g["r_lo"][t], g["r_hi"][t], g["A"][t], g["B"][t])


def test_chain_soundness_sampled():
    w = inputs.quad_chain(n_traj=2, horizon=3, n_quads=28)
    dyn = dynamics.QuadChain(28, **w.params, spring_k=w.spring_k)
    g = run_gpu(w, G=w.G)
    rng = np.random.default_rng(2)
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, G=w.G[t])
        lin = np.concatenate([g["A"][t], g["B"][t]], axis=1).astype(np.float64)
        P = np.concatenate([sampling.zonotope_points(a, w.G[t], 100000, rng),
                            sampling.box_points(lo, hi, 200000, rng)])
        R = sampling.remainders(dyn.f_batch, a, lin, P)
        assert np.all(R >= g["r_lo"][t] - 1e-15) and np.all(R <= g["r_hi"][t] + 1e-15)


def test_full_size_sampled_parity():
    """The 256-trajectory x 50-step chain of the benchmark (T = 12800, 224 x 336 generators), in the
    benchmark's launch configuration; sampled timesteps against the oracle one by one."""
    w = inputs.quad_chain(n_traj=256, horizon=50)
    dyn = dynamics.QuadChain(28, **w.params, spring_k=w.spring_k)
    h = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
    g = run_gpu(w, G=w.G, handle=h)
    assert g["flags"][0] == 0
    rng = np.random.default_rng(3)
    for t in sorted(rng.choice(w.T, 40, replace=False).tolist()) + [0, w.T - 1]:
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, G=w.G[t])
        check_parity(dyn, a, lo, hi, g["r_lo"][t], g["r_hi"][t], g["A"][t], g["B"][t])


def test_uneven_dimension_packed_batch_matches_separate_calls():
    """Chains of different length in one launch (packed rows) give the same bits as separate handles."""
    nqs = [28, 5, 1, 12]
    horizons = [4, 6, 3, 5]
    parts = [inputs.quad_chain(seed=2000 + i, n_traj=1, horizon=hz, n_quads=nq) for i, (nq, hz) in
             enumerate(zip(nqs, horizons))]
    X = np.concatenate([p.x_nom.reshape(-1) for p in parts])
    U = np.concatenate([p.u_nom.reshape(-1) for p in parts])
    G = np.concatenate([p.G.reshape(-1) for p in parts])
    offs = np.concatenate([[0], np.cumsum(horizons)]).astype(np.int32)
    h = binding.quad_chain(28, **parts[0].params, spring_k=0.5)
    out = h.bounds(_t(X), _t(U), G=_t(G), traj_offsets=_t(offs, torch.int32),
                   traj_nquads=_t(np.array(nqs, np.int32), torch.int32), n_gen_per_quad=12)
    torch.cuda.synchronize()
    rl, Al = out["r_lo"].cpu().numpy(), out["A"].cpu().numpy()
    ro = ao = 0
    for p, nq in zip(parts, nqs):
        single = run_gpu(p, G=p.G)
        n_r = single["r_lo"].size
        n_a = single["A"].size
        assert np.array_equal(rl[ro:ro + n_r], single["r_lo"].reshape(-1))
        assert np.array_equal(Al[ao:ao + n_a], single["A"].reshape(-1))
        ro += n_r
        ao += n_a
    assert ro == rl.size and ao == Al.size


def test_edge_cases():
    w = inputs.planar_quad(N=4)
    h = binding.quad_chain(1, **w.params)
    # empty batch
    out = h.bounds(_t(w.x_nom[:0]), _t(w.u_nom[:0]), radii=_t(w.radii[:0]))
    assert out["r_lo"].numel() == 0
    # non-finite input -> [-inf, inf] for that timestep only, flag raised
    rad = w.radii.copy()
    rad[2, 3] = np.nan
    g = run_gpu(w, radii=rad)
    assert g["flags"][0] & binding.ASYNC_NONFINITE
    assert np.all(np.isneginf(g["r_lo"][2])) and np.all(np.isposinf(g["r_hi"][2]))
    assert np.all(np.isfinite(g["r_lo"][[0, 1, 3]]))
    # zero radii: curved terms vanish; only the Jacobian-rounding term remains (tiny)
    g0 = run_gpu(w, radii=np.zeros_like(w.radii))
    assert np.all(np.abs(g0["r_lo"]) <= 1e-12) and np.all(np.abs(g0["r_hi"]) <= 1e-12)
    # nominal outside the set (centre offset): hull with the nominal, as the oracle
    dyn = dynamics.QuadChain(1, **w.params)
    center = w.nominal() + 0.3 * w.radii * np.sign(np.sin(np.arange(8)))[None, :] * 5
    gc = run_gpu(w, radii=w.radii, center=center.astype(np.float32))
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t], center=center.astype(np.float32)[t])
        check_parity(dyn, a, lo, hi, gc["r_lo"][t], gc["r_hi"][t])
    # a set wider than 2 pi in the angle: trig enclosures saturate to [-1, 1], still sound
    big = w.radii.copy()
    big[:, 2] = 4.0
    gb = run_gpu(w, radii=big)
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=big[t])
        check_parity(dyn, a, lo, hi, gb["r_lo"][t], gb["r_hi"][t])
    # A/B not requested: same bounds
    gn = run_gpu(w, radii=w.radii, want_AB=False)
    gy = run_gpu(w, radii=w.radii)
    assert np.array_equal(gn["r_lo"], gy["r_lo"]) and np.array_equal(gn["r_hi"], gy["r_hi"])


def test_invalid_arguments_rejected_on_host():
    w = inputs.planar_quad(N=2)
    h = binding.quad_chain(1, **w.params)
    with pytest.raises(binding.LebError):
        h.bounds(_t(w.x_nom), _t(w.u_nom))                        # box set without radii
    import ctypes as C
    bad = binding.DynamicsSpec(binding.DYN_QUAD_CHAIN, 0, 0.05, 1, 0.01, 0.1, 9.81, 0, 0, None, None, None, 0, 0, 0)
    hh = C.c_void_p()
    assert binding.lib().leb_create(C.byref(bad), C.byref(hh)) == -1    # zero quadrotors


def test_all_plans_bit_identical_and_autotune():
    w = inputs.quad_chain(n_traj=3, horizon=4, n_quads=28)
    h = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
    ref = run_gpu(w, G=w.G, handle=h)
    for i in range(h.plan_count()):
        h.select_plan(i)
        g = run_gpu(w, G=w.G, handle=h)
        for k in ("r_lo", "r_hi", "A", "B"):
            assert np.array_equal(g[k], ref[k]), (i, k)
    h.select_plan(-1)
    import tempfile, os
    with tempfile.TemporaryDirectory() as d:
        cache = os.path.join(d, "plans.txt")
        h.autotune(512, binding.SET_ZONO, 336, cache)
        assert "autotune=measured" in h.plan()
        h2 = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
        h2.autotune(512, binding.SET_ZONO, 336, cache)
        assert "autotune=cache" in h2.plan()
        g = run_gpu(w, G=w.G, handle=h)
        assert np.array_equal(g["r_lo"], ref["r_lo"])


def test_graph_capture_matches_direct_call():
    w = inputs.quad_chain(n_traj=2, horizon=5, n_quads=28)
    h = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
    ref = run_gpu(w, G=w.G, handle=h)
    x, u, G = _t(w.x_nom), _t(w.u_nom), _t(w.G)
    gr = binding.Graph(h, x, u, G=G)
    for _ in range(3):
        out = gr.launch()
    torch.cuda.synchronize()
    assert np.array_equal(out["r_lo"].cpu().numpy(), ref["r_lo"])
    assert np.array_equal(out["A"].cpu().numpy(), ref["A"])


def test_gamma_map_outputs():
    w = inputs.planar_quad()
    g = run_gpu(w, radii=w.radii, gamma_pad=1e-6)
    lo, hi = g["r_lo"], g["r_hi"]
    c, r = g["gamma_c"].reshape(lo.shape), g["gamma_r"].reshape(lo.shape)
    assert np.all(c.astype(np.float64) - r <= lo) and np.all(c.astype(np.float64) + r >= hi)
    assert np.all(r >= 1e-6)
    oc, orad = pbh.gamma_map(lo, hi, 1e-6)
    assert np.allclose(c, oc, rtol=1e-6, atol=1e-12) and np.allclose(r, orad, rtol=1e-5, atol=1e-12)
    c2, r2 = binding.zonotope_map(_t(lo), _t(hi), 1e-6)
    assert np.array_equal(c2.cpu().numpy(), c) and np.array_equal(r2.cpu().numpy(), r)


def test_zonotope_kernel_with_only_A_or_only_B():
    """The zonotope kernel's A/B writer with one of the two matrices requested: the same bounds, and the
    requested matrix identical to the one a call with both writes."""
    import ctypes as C
    w = inputs.quad_chain(n_traj=3, horizon=(2, 5), n_quads=28)
    h = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
    x, u, G = _t(w.x_nom), _t(w.u_nom), _t(w.G)
    full = h.bounds(x, u, G=G)
    torch.cuda.synchronize()
    sd = h.set_desc(G=G)
    for keep in ("A", "B"):
        lo, hi = torch.empty_like(full["r_lo"]), torch.empty_like(full["r_hi"])
        mat = torch.full_like(full[keep], float("nan"))
        flags = torch.zeros(1, device=DEV, dtype=torch.int32)
        ws = h.workspace(w.T)
        ptr = binding._ptr
        st = binding.lib().leb_bounds(h.h, None, w.T, ptr(x), ptr(u), C.byref(sd), ptr(lo), ptr(hi),
                                      ptr(mat) if keep == "A" else None, ptr(mat) if keep == "B" else None, None,
                                      ptr(ws), ws.numel(), ptr(flags), binding._stream())
        binding.check(st, "leb_bounds")
        torch.cuda.synchronize()
        assert int(flags.item()) == 0
        assert torch.equal(lo, full["r_lo"]) and torch.equal(hi, full["r_hi"])
        assert torch.equal(mat, full[keep]), keep


def test_inputs_first_path_order_parity():
    """Thm. 1 with the path taking the inputs first (leb_set_path_order): every timestep of the planar
    quadrotor (box sets) and of a ragged 28-quadrotor chain batch (zonotope sets) against the oracle with
    the same order; the adjoint and the nominal refinement refuse that order."""
    w = inputs.planar_quad()
    dyn = dynamics.QuadChain(1, **w.params)
    order = list(range(6, 8)) + list(range(6))
    h = binding.quad_chain(1, **w.params)
    h.set_path_order(True)
    g = run_gpu(w, radii=w.radii, handle=h)
    gn = run_gpu(w, radii=w.radii)
    assert g["flags"][0] == 0
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        ol, oh = pbh.pbh(dyn, a, lo, hi, order=order)
        J = dyn.jacobian(a)
        eps = tolerance(dyn, a, lo, hi, J)
        scale = np.abs(ol) + np.abs(oh) + 1e-300
        assert np.all(g["r_lo"][t] <= ol + 1e-12 * scale) and np.all(g["r_hi"][t] >= oh - 1e-12 * scale)
        assert np.all((g["r_hi"][t] - g["r_lo"][t]) <= (oh - ol) * (1 + 1e-5) + eps)
    assert np.array_equal(g["A"], gn["A"]) and np.array_equal(g["B"], gn["B"])
    # the order the paper's systems favour: tighter on average than the natural one here too
    assert (g["r_hi"] - g["r_lo"]).sum() < (gn["r_hi"] - gn["r_lo"]).sum()
    with pytest.raises(binding.LebError):
        h.bounds_backward(_t(w.x_nom), _t(w.u_nom), _t(w.radii), _t(np.ones((w.T, 6))), _t(np.ones((w.T, 6))))
    # ragged chain batch, zonotope sets (the stream kernel)
    wc = inputs.quad_chain(n_traj=3, horizon=(2, 6), n_quads=28)
    dc = dynamics.QuadChain(28, **wc.params, spring_k=wc.spring_k)
    hc = binding.quad_chain(28, **wc.params, spring_k=wc.spring_k)
    hc.set_path_order(True)
    gc = run_gpu(wc, G=wc.G, batch=True, handle=hc)
    oc = list(range(168, 224)) + list(range(168))
    for t in range(wc.T):
        a = wc.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, G=wc.G[t])
        ol, oh = pbh.pbh(dc, a, lo, hi, order=oc)
        eps = tolerance(dc, a, lo, hi, dc.jacobian(a))
        scale = np.abs(ol) + np.abs(oh) + 1e-300
        assert np.all(gc["r_lo"][t] <= ol + 1e-12 * scale) and np.all(gc["r_hi"][t] >= oh - 1e-12 * scale)
        assert np.all((gc["r_hi"][t] - gc["r_lo"][t]) <= (oh - ol) * (1 + 1e-5) + eps)


def test_attitude_partition_parity():
    """Input-domain partitioning (leb_set_partition): every quadrotor's attitude box cut at the nominal,
    Thm. 1 on each piece, the hull; against the oracle's partitioned bound on every timestep of the planar
    quadrotor and of two coupled quadrotors, inside the plain GPU bound."""
    cases = []
    w = inputs.planar_quad()
    cases.append((w, dynamics.QuadChain(1, **w.params), dict(radii=w.radii), [2]))
    w2 = inputs.quad_chain(n_traj=2, horizon=4, n_quads=2)
    cases.append((w2, dynamics.QuadChain(2, **w2.params, spring_k=w2.spring_k), dict(G=w2.G, batch=True), [2, 8]))
    for wk, dyn, kw, dims in cases:
        h = binding.quad_chain(wk.n_quads, **wk.params, spring_k=wk.spring_k)
        h.set_partition(True)
        g = run_gpu(wk, handle=h, **kw)
        gp = run_gpu(wk, **kw)
        assert g["flags"][0] == 0
        assert np.all(g["r_lo"] >= gp["r_lo"]) and np.all(g["r_hi"] <= gp["r_hi"])
        assert np.array_equal(g["A"], gp["A"]) and np.array_equal(g["B"], gp["B"])
        for t in range(wk.T):
            a = wk.nominal()[t].astype(np.float64)
            if "G" in kw:
                lo, hi = pbh.box_from_set(a, G=wk.G[t])
            else:
                lo, hi = pbh.box_from_set(a, radii=wk.radii[t])
            ol, oh = pbh.pbh_partitioned(dyn, a, lo, hi, dims)
            eps = tolerance(dyn, a, lo, hi, dyn.jacobian(a))
            scale = np.abs(ol) + np.abs(oh) + 1e-300
            assert np.all(g["r_lo"][t] <= ol + 1e-12 * scale) and np.all(g["r_hi"][t] >= oh - 1e-12 * scale)
            assert np.all((g["r_hi"][t] - g["r_lo"][t]) <= (oh - ol) * (1 + 1e-5) + eps)
    with pytest.raises(binding.LebError):
        h.bounds_backward(_t(w2.x_nom), _t(w2.u_nom), _t(np.full((w2.T, 16), 0.05, np.float32)),
                          _t(np.ones((w2.T, 12))), _t(np.ones((w2.T, 12))))


def recentred_tolerance(dyn, a, lo, hi, J):
    """The plain bound's FP32 tolerance plus, per curved row, the enclosure slack of the re-centred terms:
    the point remainder at beta (a difference of two sin or cos enclosures, each within 2^-22 of the value,
    times (dt/m) S, plus the rounding of A (beta - alpha~)) and the Jacobian at beta (its sin/cos
    enclosures times the piece's displacements)."""
    eps = tolerance(dyn, a, lo, hi, J)
    D = np.maximum(np.abs(lo - a), np.abs(hi - a))
    c = dyn.dt / dyn.m
    for i in range(dyn.nq):
        jp, j1, j2 = dyn.ix(i, 2), dyn.n_x + 2 * i, dyn.n_x + 2 * i + 1
        Smax = abs(a[j1]) + abs(a[j2]) + D[j1] + D[j2]
        slack = c * Smax * 8 * 2.0 ** -22 + 4 * 2.0 ** -22 * c * (Smax * D[jp] + D[j1] + D[j2])
        slack += 2.0 ** -22 * (np.abs(J[dyn.ix(i, 3)]).max() + np.abs(J[dyn.ix(i, 4)]).max()) * D[jp]
        eps[dyn.ix(i, 3)] += slack
        eps[dyn.ix(i, 4)] += slack
    return eps


@pytest.mark.parametrize("pieces", [4, 16])
def test_recentred_partition_parity(pieces):
    """Re-centred input-domain partitioning (leb_set_partition_recentred): each attitude box in equal
    pieces expanded around their midpoints, against the oracle's pbh_recentred with the same pieces and
    the returned A, on every timestep of the planar quadrotor (box sets) and of a ragged batch of two
    coupled quadrotors (zonotope hulls); A and B are those of the plain call. The planar quadrotor's
    bounds also contain its exact remainder range and are narrower than the plain ones."""
    from oracle import exact
    cases = []
    w = inputs.planar_quad()
    cases.append((w, dynamics.QuadChain(1, **w.params), dict(radii=w.radii)))
    w2 = inputs.quad_chain(n_traj=2, horizon=4, n_quads=2)
    cases.append((w2, dynamics.QuadChain(2, **w2.params, spring_k=w2.spring_k), dict(G=w2.G, batch=True)))
    for wk, dyn, kw in cases:
        h = binding.quad_chain(wk.n_quads, **wk.params, spring_k=wk.spring_k)
        h.set_partition_recentred(pieces)
        g = run_gpu(wk, handle=h, **kw)
        gp = run_gpu(wk, **kw)
        assert g["flags"][0] == 0
        assert np.array_equal(g["A"], gp["A"]) and np.array_equal(g["B"], gp["B"])
        dims = [dyn.ix(i, 2) for i in range(dyn.nq)]
        for t in range(wk.T):
            a = wk.nominal()[t].astype(np.float64)
            lo, hi = pbh.box_from_set(a, G=wk.G[t]) if "G" in kw else pbh.box_from_set(a, radii=wk.radii[t])
            AB = np.concatenate([g["A"][t], g["B"][t]], axis=1).astype(np.float64)
            ol, oh = pbh.pbh_recentred(dyn, a, lo, hi, dims, pieces, A=AB)
            eps = recentred_tolerance(dyn, a, lo, hi, dyn.jacobian(a))
            scale = np.abs(ol) + np.abs(oh) + 1e-300
            assert np.all(g["r_lo"][t] <= ol + 1e-12 * scale), (t, np.max(g["r_lo"][t] - ol))
            assert np.all(g["r_hi"][t] >= oh - 1e-12 * scale), (t, np.max(oh - g["r_hi"][t]))
            assert np.all((g["r_hi"][t] - g["r_lo"][t]) <= (oh - ol) * (1 + 1e-5) + eps)
            if dyn.nq == 1:
                el, eh = exact.quad_exact_range(dyn, a, lo, hi)
                # w.r.t. the FP32 A: the exact range moves by at most (J - A) Delta
                d = np.abs(dyn.jacobian(a) - AB) @ np.maximum(np.abs(lo - a), np.abs(hi - a))
                assert np.all(g["r_lo"][t] <= el + d + 1e-12) and np.all(g["r_hi"][t] >= eh - d - 1e-12)
        ratio = (g["r_hi"] - g["r_lo"]).sum() / (gp["r_hi"] - gp["r_lo"]).sum()
        print(f"re-centred partition, {pieces} pieces, {dyn.nq} quadrotor(s): width / plain = {ratio:.4f}")
        if dyn.nq == 1:
            assert ratio < 1.0


def test_recentred_partition_full_size_sampled():
    """The benchmark's 256 x 50 chain of 28 quadrotors (zonotope 224 x 336) with 8 re-centred pieces per
    attitude, in the benchmark's launch configuration (the persistent TMA kernel); sampled timesteps
    against the oracle one by one."""
    w = inputs.quad_chain(n_traj=256, horizon=50)
    dyn = dynamics.QuadChain(28, **w.params, spring_k=w.spring_k)
    h = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
    h.set_partition_recentred(8)
    g = run_gpu(w, G=w.G, handle=h)
    assert g["flags"][0] == 0
    dims = [dyn.ix(i, 2) for i in range(28)]
    rng = np.random.default_rng(4)
    for t in sorted(rng.choice(w.T, 12, replace=False).tolist()) + [w.T - 1]:
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, G=w.G[t])
        AB = np.concatenate([g["A"][t], g["B"][t]], axis=1).astype(np.float64)
        ol, oh = pbh.pbh_recentred(dyn, a, lo, hi, dims, 8, A=AB)
        eps = recentred_tolerance(dyn, a, lo, hi, dyn.jacobian(a))
        scale = np.abs(ol) + np.abs(oh) + 1e-300
        assert np.all(g["r_lo"][t] <= ol + 1e-12 * scale) and np.all(g["r_hi"][t] >= oh - 1e-12 * scale), t
        assert np.all((g["r_hi"][t] - g["r_lo"][t]) <= (oh - ol) * (1 + 1e-5) + eps), t
