"""GPU parity of the path-based Hessian bound (Thm. 1) for the paper's satellite and (coupled) 3-D
quadrotor models (App. A) against the FP64 oracle, through the C ABI.

Tolerance (from the kernel's FP32 arithmetic): the GPU interval encloses the same Eq. 15, term for term
the same interval expressions, on an outward-rounded hull, plus (J - A) Delta for the FP32 Jacobian it
returns. Per row l:
  * containment: gpu_lo <= oracle_lo + 1e-12 s_l and gpu_hi >= oracle_hi - 1e-12 s_l;
  * width: gpu_w <= oracle_w (1 + 1e-5) + eps_l with
        eps_l = 2^-18 sum_terms Hm D_j D_k + 2 sum_terms Hm ((D_j + d_j)(D_k + d_k) - D_j D_k)
                + 2^-20 max_k |J_lk| sum_{j in row} D_j,
    Hm the entry's interval magnitude over the box with every angle widened by 0.5 (4 for roll and yaw),
    which bounds the absolute slack of the sin / cos / tan / sec enclosures, d_j = 2^-22 (|alpha~_j| + D_j)
    the widening from storing the box ends as outward-rounded FP32, and the last term the rounding of the
    Jacobian entries (every row of an Euler step has a diagonal entry near 1, so max_k |J_lk| bounds the
    scale of the trigonometric slack in the row's Jacobian).
A is checked against the FP64 Jacobian to 2^-21 (|J| + max_k |J_lk|).
"""
import math

import numpy as np
import pytest
import torch

from oracle import dynamics3d, pbh, sampling
from paper_2607_01203_b300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _t(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV, dtype)


def _pair(w):
    if w.kind == "satellite":
        return binding.satellite(**w.params), dynamics3d.Satellite(**w.params)
    return binding.quad3d(w.n_quads, **w.params), dynamics3d.Quad3D(w.n_quads, **w.params)


def run_gpu(h, w, center=None, want_AB=True, **kw):
    out = h.bounds(_t(w.x_nom), _t(w.u_nom), radii=_t(w.radii), center=None if center is None else _t(center),
                   want_AB=want_AB, **kw)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


def _widened(dyn, lo, hi):
    wl, wh = lo.copy(), hi.copy()
    if isinstance(dyn, dynamics3d.Quad3D):
        for i in range(dyn.nq):
            for s, pad in ((3, 4.0), (4, 0.5), (5, 4.0)):
                j = dyn.ix(i, s)
                wl[j], wh[j] = lo[j] - pad, hi[j] + pad
    return wl, wh


def tolerance(dyn, a, lo, hi, J):
    D = np.maximum(np.abs(lo - a), np.abs(hi - a))
    dD = 2.0 ** -22 * (np.abs(a) + D)
    wl, wh = _widened(dyn, lo, hi)
    eps = 2.0 ** -20 * np.abs(J).max(axis=1) * ((J != 0) @ D)
    for row in range(dyn.n_x):
        for j, k, fn in dyn.hessian_terms(row):
            Hm = max(abs(v) for v in fn(wl, wh))
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
        AB = np.concatenate([A, B], axis=1).astype(np.float64)
        tolJ = 2.0 ** -21 * (np.abs(J) + np.abs(J).max(axis=1, keepdims=True))
        assert np.all(np.abs(AB - J) <= tolJ), np.max(np.abs(AB - J) - tolJ)
    return ol, oh


def test_tan_sec_enclosures_contain_fp64_values():
    lib = binding.lib()
    rng = np.random.default_rng(60)
    edge = np.float32(1.5707)
    x = np.concatenate([rng.uniform(-1.5, 1.5, 200000), rng.uniform(-1.5707, 1.5707, 100000),
                        rng.normal(size=20000) * 1e-3,
                        [0.0, -0.0, 1e-40, -1e-40, 1e-7, 0.7853982, 1.0, 1.5, 1.57,
                         np.nextafter(edge, np.float32(0)), -np.nextafter(edge, np.float32(0))]]).astype(np.float32)
    xt = _t(x)
    out = [torch.empty(x.size, 2, device=DEV) for _ in range(2)]
    binding.check(lib.leb_selftest_tan_sec(xt.data_ptr(), x.size, out[0].data_ptr(), out[1].data_ptr(), None),
                  "selftest")
    torch.cuda.synchronize()
    xd = x.astype(np.float64)
    sec = 1.0 / np.cos(xd)
    # tan: 8 ulps of the value on each side; sec = 1 / cos: the absolute slack 2^-22 of the cos enclosure
    # becomes 2^-21 sec^2 in width, plus the rounding of the reciprocals; within the cos enclosure's
    # extremum margin m = 2e-3 + 4e-7 |x| of 0 its upper end is raised to 1 (at most m^2 / 2 higher)
    m = 2e-3 + 4e-7 * np.abs(xd)
    for enc, ref, tol in ((out[0], np.tan(xd), 2.0 ** -18 * np.abs(np.tan(xd)) + 1e-37),
                          (out[1], sec, (2.0 ** -20 + np.where(np.abs(xd) < m, m * m, 0.0)) * sec ** 2
                           + 2.0 ** -21 * sec)):
        e = enc.cpu().numpy().astype(np.float64)
        assert np.all(e[:, 0] <= ref) and np.all(e[:, 1] >= ref)
        assert np.all(e[:, 1] - e[:, 0] <= tol)
    # outside the domain (and at its edge) the enclosure is the whole line
    bad = _t(np.array([1.5707, -1.5707, 1.6, -2.0, 3.0, np.nan], np.float32))
    o2 = [torch.empty(6, 2, device=DEV) for _ in range(2)]
    binding.check(lib.leb_selftest_tan_sec(bad.data_ptr(), 6, o2[0].data_ptr(), o2[1].data_ptr(), None), "selftest")
    torch.cuda.synchronize()
    for e in o2:
        e = e.cpu().numpy()
        assert np.all(e[:, 0] == -np.inf) and np.all(e[:, 1] == np.inf)


@pytest.mark.parametrize("eps", [0.01, 0.1, 0.2])
def test_satellite_parity_all_timesteps(eps):
    w = inputs.satellite(T=301, eps=eps)     # 8 full groups of 36 timesteps and a ragged tail of 13
    h, dyn = _pair(w)
    g = run_gpu(h, w)
    assert g["flags"][0] == 0
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        check_parity(dyn, a, lo, hi, g["r_lo"][t], g["r_hi"][t], g["A"][t], g["B"][t])


@pytest.mark.parametrize("nq,coupled,eps", [(1, False, 0.01), (1, False, 0.2), (3, True, 0.05), (2, False, 0.1)])
def test_quad3d_parity_all_timesteps(nq, coupled, eps):
    w = inputs.quad3d(T=50, n_quads=nq, eps=eps, coupled=coupled)
    h, dyn = _pair(w)
    g = run_gpu(h, w)
    assert g["flags"][0] == 0
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        check_parity(dyn, a, lo, hi, g["r_lo"][t], g["r_hi"][t], g["A"][t], g["B"][t])


def test_coupled_168d_parity_sampled():
    """The paper's 168-state system: 14 coupled 3-D quadrotors, 64 trajectories of horizon 25 in one launch,
    sampled timesteps against the oracle one by one."""
    w = inputs.quad3d(T=64 * 25, n_quads=14, eps=0.05, coupled=True, N=25)
    h, dyn = _pair(w)
    g = run_gpu(h, w)
    assert g["flags"][0] == 0
    rng = np.random.default_rng(61)
    for t in sorted(rng.choice(w.T, 5, replace=False).tolist()) + [w.T - 1]:
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        check_parity(dyn, a, lo, hi, g["r_lo"][t], g["r_hi"][t], g["A"][t], g["B"][t])


def test_max_quadrotors_and_centre_offset():
    """21 quadrotors (252 rows, the largest one CTA holds) with a set centred away from the nominal."""
    w = inputs.quad3d(T=7, n_quads=21, eps=0.03, coupled=True)
    h, dyn = _pair(w)
    rng = np.random.default_rng(62)
    center = w.nominal() + rng.uniform(-0.02, 0.02, w.nominal().shape).astype(np.float32)
    g = run_gpu(h, w, center=center)
    assert g["flags"][0] == 0
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t], center=center[t].astype(np.float64))
        check_parity(dyn, a, lo, hi, g["r_lo"][t], g["r_hi"][t], g["A"][t], g["B"][t])
    with pytest.raises(binding.LebError):
        binding.quad3d(22, **inputs.QUAD3D)


@pytest.mark.parametrize("which", ["satellite", "quad3d", "coupled"])
def test_soundness_sampled(which):
    """Zero violations of the true remainder, w.r.t. the returned FP32 A, B, over 2.5 10^5 points per set
    (box vertices and faces included)."""
    if which == "satellite":
        w = inputs.satellite(T=6, eps=0.2)
    else:
        w = inputs.quad3d(T=6, n_quads=1 if which == "quad3d" else 3, eps=0.2, coupled=which == "coupled")
    h, dyn = _pair(w)
    g = run_gpu(h, w)
    rng = np.random.default_rng(63)
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        lin = np.concatenate([g["A"][t], g["B"][t]], axis=1).astype(np.float64)
        P = sampling.box_points(lo, hi, 250000, rng)
        R = sampling.remainders(dyn.f_batch, a, lin, P)
        assert np.all(R >= g["r_lo"][t].astype(np.float64) - 2e-14)
        assert np.all(R <= g["r_hi"][t].astype(np.float64) + 2e-14)


def test_edge_cases():
    w = inputs.quad3d(T=5, n_quads=2, eps=0.05)
    h, dyn = _pair(w)
    # T = 0: nothing to do, flags cleared
    out = h.bounds(_t(w.x_nom[:0]), _t(w.u_nom[:0]), radii=_t(w.radii[:0]))
    torch.cuda.synchronize()
    assert int(out["flags"].item()) == 0
    # zero radii: the remainder is 0 at the nominal; the bound contains it and is tiny
    w0 = inputs.quad3d(T=5, n_quads=2, eps=0.0)
    g = run_gpu(h, w0)
    assert np.all(g["r_lo"] <= 0) and np.all(g["r_hi"] >= 0) and np.all(g["r_hi"] - g["r_lo"] == 0)
    # a non-finite input poisons only its own timestep, and raises the flag
    x = w.x_nom.copy()
    x[2, 7] = np.nan
    g = h.bounds(_t(x), _t(w.u_nom), radii=_t(w.radii))
    torch.cuda.synchronize()
    assert int(g["flags"].item()) & 1
    rl, rh = g["r_lo"].cpu().numpy(), g["r_hi"].cpu().numpy()
    assert np.all(rl[2] == -np.inf) and np.all(rh[2] == np.inf)
    assert np.all(np.isfinite(rl[[0, 1, 3, 4]])) and np.all(np.isfinite(rh[[0, 1, 3, 4]]))
    # pitch box reaching the tan / sec singularity: the roll and yaw rows of that quadrotor become
    # [-inf, inf], every other row stays finite and sound
    x = w.x_nom.copy()
    x[1, 4] = 1.55
    g = run_gpu(h, dataclass_with(w, x_nom=x))
    assert g["flags"][0] == 0
    assert np.all(g["r_lo"][1, [3, 5]] == -np.inf) and np.all(g["r_hi"][1, [3, 5]] == np.inf)
    others = [l for l in range(w.n_x) if l not in (3, 5)]
    assert np.all(np.isfinite(g["r_lo"][1, others]))
    # zonotope sets and uneven batches are refused on the host
    with pytest.raises(binding.LebError):
        h.bounds(_t(w.x_nom), _t(w.u_nom), G=_t(np.zeros((w.T, w.n, 2), np.float32)))


def dataclass_with(w, **kw):
    import dataclasses
    return dataclasses.replace(w, **kw)


def test_options_static_entry_and_gamma():
    """The zonotope map outputs of Sec. IV-C, and leb_bounds_static giving the same bits as leb_bounds."""
    w = inputs.quad3d(T=100, n_quads=3, eps=0.1, coupled=True)
    h, _ = _pair(w)
    g = run_gpu(h, w, gamma_pad=1e-3, want_eps=True)
    c, r = g["gamma_c"].astype(np.float64), g["gamma_r"].astype(np.float64)
    assert np.all(c - r <= g["r_lo"]) and np.all(c + r >= g["r_hi"]) and np.all(r >= 1e-3)
    assert np.all(g["eps"] == 0)
    x, u, rad = _t(w.x_nom), _t(w.u_nom), _t(w.radii)
    rl, rh = torch.empty(w.T, w.n_x, device=DEV), torch.empty(w.T, w.n_x, device=DEV)
    A, B = torch.empty(w.T, w.n_x, w.n_x, device=DEV), torch.empty(w.T, w.n_x, w.n_u, device=DEV)
    fl = torch.ones(1, dtype=torch.int32, device=DEV)
    sd = binding.Handle.set_desc(radii=rad)
    binding.check(binding.lib().leb_bounds_static(h.h, None, w.T, x.data_ptr(), u.data_ptr(), binding.C.byref(sd),
                                                  rl.data_ptr(), rh.data_ptr(), A.data_ptr(), B.data_ptr(),
                                                  fl.data_ptr(), None), "leb_bounds_static")
    torch.cuda.synchronize()
    assert int(fl.item()) == 0
    assert np.array_equal(rl.cpu().numpy(), g["r_lo"]) and np.array_equal(rh.cpu().numpy(), g["r_hi"])
    assert np.array_equal(A.cpu().numpy(), g["A"]) and np.array_equal(B.cpu().numpy(), g["B"])


def test_pbh_is_tighter_than_interval_hessians():
    """Corollary 1 on the GPU bound: the mean width is at most that of the FP64 IH expansion (Eq. 13)
    over the same boxes, itself at most the classic interval quadratic form (Eq. 12)."""
    for w in (inputs.satellite(T=40, eps=0.2), inputs.quad3d(T=40, eps=0.2)):
        h, dyn = _pair(w)
        g = run_gpu(h, w, want_AB=False)
        wg, we, wc = 0.0, 0.0, 0.0
        for t in range(w.T):
            a = w.nominal()[t].astype(np.float64)
            lo, hi = pbh.box_from_set(a, radii=w.radii[t])
            E, C = pbh.ih_expand(dyn, a, lo, hi), pbh.ih_classic(dyn, a, lo, hi)
            wg += float((g["r_hi"][t] - g["r_lo"][t]).sum())
            we += float((E[1] - E[0]).sum())
            wc += float((C[1] - C[0]).sum())
        assert wg <= we * (1 + 1e-4) and we <= wc * (1 + 1e-12)


def test_width_vs_eps_report():
    """The width-versus-eps study of the paper's Fig. 2 on synthetic nominal points: mean interval width of
    the bound per state row for PBH (GPU), the interval-Hessian expansion (Eq. 13) and the classic
    interval quadratic form (Eq. 12) (FP64 oracle), and random sampling of 10^4 points per set (an
    under-approximation). The ordering sampling <= PBH <= IH-expand <= IH-classic holds at every eps;
    the table is printed (pytest -s) for the design notes."""
    rng = np.random.default_rng(64)
    lines = ["system     eps    sampling   PBH(gpu)   IH-expand  IH-classic"]
    for name in ("satellite", "quadrotor"):
        for eps in (0.01, 0.05, 0.1, 0.15, 0.2):
            w = inputs.satellite(T=40, eps=eps) if name == "satellite" else inputs.quad3d(T=40, eps=eps)
            h, dyn = _pair(w)
            g = run_gpu(h, w, want_AB=False)
            acc = np.zeros(4)
            for t in range(w.T):
                a = w.nominal()[t].astype(np.float64)
                lo, hi = pbh.box_from_set(a, radii=w.radii[t])
                E, C = pbh.ih_expand(dyn, a, lo, hi), pbh.ih_classic(dyn, a, lo, hi)
                R = sampling.remainders(dyn.f_batch, a, dyn.jacobian(a), sampling.box_points(lo, hi, 10000, rng))
                acc += [np.mean(R.max(0) - R.min(0)), np.mean(g["r_hi"][t] - g["r_lo"][t]),
                        np.mean(E[1] - E[0]), np.mean(C[1] - C[0])]
            acc /= w.T
            lines.append(f"{name:10s} {eps:4.2f}  " + "  ".join(f"{v:9.3e}" for v in acc))
            assert acc[0] <= acc[1] <= acc[2] * (1 + 1e-4) and acc[2] <= acc[3] * (1 + 1e-12)
    print("\n" + "\n".join(lines))


def test_graph_capture_matches_direct_call():
    """leb_graph_capture of the satellite and the 168-state coupled system: replays give the direct call's
    bits (the launch is allocation-free and capturable for these kinds too)."""
    for w in (inputs.satellite(T=333, eps=0.1), inputs.quad3d(T=3 * 25, n_quads=14, eps=0.05, coupled=True, N=25)):
        h, _ = _pair(w)
        ref = run_gpu(h, w)
        x, u, r = _t(w.x_nom), _t(w.u_nom), _t(w.radii)
        gr = binding.Graph(h, x, u, radii=r)
        for _ in range(3):
            out = gr.launch()
        torch.cuda.synchronize()
        assert int(out["flags"].item()) == 0
        for k in ("r_lo", "r_hi", "A", "B"):
            assert np.array_equal(out[k].cpu().numpy(), ref[k]), k


def _global_order(dyn, local):
    """The path order over all coordinates of a (coupled) 3-D quadrotor system given each quadrotor's
    local order (states 0..11, inputs 12..15): quadrotor by quadrotor, each in its local order (only the
    relative order of a quadrotor's own coordinates matters to its rows)."""
    g = []
    for i in range(dyn.nq):
        for c in local:
            g.append(12 * i + c if c < 12 else 12 * dyn.nq + 4 * i + (c - 12))
    return g


def _angle_orders():
    """The 12 orders of the path-order study: the three angles in any order, the thrust first or last, the
    other coordinates in their natural places."""
    import itertools
    out = []
    for perm in itertools.permutations((3, 4, 5)):
        nat = [0, 1, 2] + list(perm) + [6, 7, 8, 9, 10, 11, 12, 13, 14, 15]
        out.append(nat)
        out.append([12] + [c for c in nat if c != 12])
    return out


def test_general_path_order_parity():
    """leb_set_path_order_perm on the 3-D quadrotor: for the 12 orders of the study (angle orders, thrust
    first or last) and random permutations of all 16 coordinates, the GPU bounds against the oracle's Thm. 1
    with the same order (each entry over the prefix set of its first coordinate), on single and three
    coupled quadrotors; A and B do not depend on the order. The best of the 12 is reported against the
    natural order on the E1 points."""
    rng = np.random.default_rng(61)
    orders = _angle_orders() + [list(rng.permutation(16)) for _ in range(4)]
    assert len({tuple(o) for o in orders[:12]}) == 12
    for nq, coupled in ((1, False), (3, True)):
        w = inputs.quad3d(T=24, n_quads=nq, eps=0.1, coupled=coupled)
        h, dyn = _pair(w)
        plain = run_gpu(h, w)
        widths = []
        for od in orders:
            h.set_path_order_perm(od)
            g = run_gpu(h, w)
            assert g["flags"][0] == 0
            assert np.array_equal(g["A"], plain["A"]) and np.array_equal(g["B"], plain["B"])
            go = _global_order(dyn, od)
            for t in range(w.T):
                a = w.nominal()[t].astype(np.float64)
                lo, hi = pbh.box_from_set(a, radii=w.radii[t], center=None)
                ol, oh = pbh.pbh(dyn, a, lo, hi, order=go)
                eps = tolerance(dyn, a, lo, hi, dyn.jacobian(a))
                scale = np.abs(ol) + np.abs(oh) + 1e-300
                gl, gh = g["r_lo"][t].astype(np.float64), g["r_hi"][t].astype(np.float64)
                assert np.all(gl <= ol + 1e-12 * scale) and np.all(gh >= oh - 1e-12 * scale), (od, t)
                assert np.all((gh - gl) <= (oh - ol) * (1 + 1e-5) + eps), (od, t)
            widths.append(float((g["r_hi"] - g["r_lo"]).mean()))
        h.set_path_order_perm(None)
        g = run_gpu(h, w)
        assert np.array_equal(g["r_lo"], plain["r_lo"]) and np.array_equal(g["r_hi"], plain["r_hi"])
        nat = float((plain["r_hi"] - plain["r_lo"]).mean())
        best = int(np.argmin(widths[:12]))
        print(f"{nq} quadrotor(s): best of the 12 orders {orders[best]} width / natural = {widths[best] / nat:.4f}")
    with pytest.raises(binding.LebError):
        h.set_path_order_perm([0] * 16)
    with pytest.raises(binding.LebError):
        h.set_path_order_perm(list(range(15)))


def test_chain_general_path_order_parity():
    """The quad chain with one input before the attitude and the other after it (a local order that
    leb_set_path_order cannot express), against the oracle's Thm. 1 with that order, every timestep of a
    two-quadrotor zonotope batch."""
    from oracle import dynamics
    import test_gpu_pbh as tp
    w = inputs.quad_chain(n_traj=2, horizon=4, n_quads=2)
    dyn = dynamics.QuadChain(2, **w.params, spring_k=w.spring_k)
    h = binding.quad_chain(2, **w.params, spring_k=w.spring_k)
    local = [0, 1, 7, 3, 2, 4, 5, 6]        # u2 before phi, u1 after
    h.set_path_order_perm(local)
    g = tp.run_gpu(w, G=w.G, handle=h, batch=True)
    assert g["flags"][0] == 0
    go = []
    for i in range(2):
        for c in local:
            go.append(6 * i + c if c < 6 else 12 + 2 * i + (c - 6))
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, G=w.G[t])
        ol, oh = pbh.pbh(dyn, a, lo, hi, order=go)
        eps = tp.tolerance(dyn, a, lo, hi, dyn.jacobian(a))
        scale = np.abs(ol) + np.abs(oh) + 1e-300
        assert np.all(g["r_lo"][t] <= ol + 1e-12 * scale) and np.all(g["r_hi"][t] >= oh - 1e-12 * scale), t
        assert np.all((g["r_hi"][t] - g["r_lo"][t]) <= (oh - ol) * (1 + 1e-5) + eps), t
