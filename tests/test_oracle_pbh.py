"""Pins of the FP64 PBH oracle (Thm. 1) against things other than itself (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import dynamics, exact, pbh, sampling
from paper_2607_01203_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def quad():
    w = inputs.planar_quad()
    return w, dynamics.QuadChain(1, **w.params)


def test_jacobian_matches_finite_differences(quad):
    """Eq. 8 entries hand-derived from App. A vs central differences of f."""
    w, dyn = quad
    chain = dynamics.QuadChain(4, **w.params, spring_k=0.5)
    rng = np.random.default_rng(0)
    for d in (dyn, chain):
        for _ in range(5):
            a = rng.normal(size=d.n) * 2
            Jfd = np.zeros((d.n_x, d.n))
            for i in range(d.n):
                e = np.zeros(d.n)
                e[i] = 1e-6
                Jfd[:, i] = (d.f(a + e) - d.f(a - e)) / 2e-6
            assert np.abs(Jfd - d.jacobian(a)).max() < 1e-7


def test_hessian_table_matches_finite_differences(quad):
    """Every hand-derived second derivative, and the absence of others, vs differences of the Jacobian."""
    w, dyn = quad
    chain = dynamics.QuadChain(3, **w.params, spring_k=0.5)
    rng = np.random.default_rng(1)
    for d in (dyn, chain):
        for _ in range(4):
            a = rng.normal(size=d.n) * 2
            H = d.hessian_point(a)
            Hfd = np.zeros_like(H)
            for i in range(d.n):
                e = np.zeros(d.n)
                e[i] = 1e-5
                Hfd[:, :, i] = (d.jacobian(a + e) - d.jacobian(a - e)) / 2e-5
            assert np.abs(H - Hfd).max() < 1e-7


def test_worked_example_golden(quad):
    """Hand evaluation of Eq. 15 (tests/golden/pbh_worked_example.txt)."""
    w, dyn = quad
    a = np.zeros(8)
    a[6] = a[7] = 5.0
    lo = a.copy()
    hi = a.copy()
    lo[2], hi[2] = -0.1, 0.1
    lo[6:], hi[6:] = 4.5, 5.5
    Rl, Rh = pbh.pbh(dyn, a, lo, hi)
    rows = np.loadtxt(os.path.join(GOLDEN, "pbh_worked_example.txt"))
    for row, glo, ghi in rows:
        assert Rl[int(row)] == pytest.approx(glo, abs=1e-15)
        assert Rh[int(row)] == pytest.approx(ghi, abs=1e-15)
    others = [r for r in range(6) if r not in (3, 4)]
    assert np.all(Rl[others] == 0) and np.all(Rh[others] == 0)


def test_contains_exact_range_planar_quad(quad):
    """Thm. 1 soundness: PBH contains the exact remainder range on every timestep of the workload."""
    w, dyn = quad
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        Rl, Rh = pbh.pbh(dyn, a, lo, hi)
        El, Eh = exact.quad_exact_range(dyn, a, lo, hi)
        assert np.all(Rl <= El + 1e-15) and np.all(Rh >= Eh - 1e-15)
        # tight to a constant factor: the curved rows' widths stay within 3x of exact
        for r in (3, 4):
            assert (Rh[r] - Rl[r]) <= 3.0 * (Eh[r] - El[r]) + 1e-12


def test_exact_range_matches_brute_force(quad):
    """The exact-range oracle itself against dense sampling of the true remainder (incl. vertices)."""
    w, dyn = quad
    rng = np.random.default_rng(2)
    for t in (0, 7, 13):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        El, Eh = exact.quad_exact_range(dyn, a, lo, hi)
        P = sampling.box_points(lo, hi, 60000, rng)
        R = sampling.remainders(dyn.f_batch, a, dyn.jacobian(a), P)
        assert np.all(R.min(0) >= El - 1e-14) and np.all(R.max(0) <= Eh + 1e-14)
        for r in (3, 4):    # vertices attain the extremes up to sampling
            assert R.min(0)[r] <= El[r] + 0.02 * (Eh[r] - El[r])
            assert R.max(0)[r] >= Eh[r] - 0.02 * (Eh[r] - El[r])


def test_corollary1_ordering(quad):
    """Cor. 1: for symmetric Delta, R_path within R_expand within R_classic."""
    w, dyn = quad
    rng = np.random.default_rng(3)
    for _ in range(30):
        a = np.concatenate([rng.normal(size=6) * 3, rng.uniform(3, 7, 2)])
        rad = rng.uniform(0.01, 0.5, 8)
        lo, hi = a - rad, a + rad
        P = pbh.pbh(dyn, a, lo, hi)
        E = pbh.ih_expand(dyn, a, lo, hi)
        C = pbh.ih_classic(dyn, a, lo, hi)
        assert np.all(E[0] <= P[0] + 1e-15) and np.all(P[1] <= E[1] + 1e-15)
        assert np.all(C[0] <= E[0] + 1e-15) and np.all(E[1] <= C[1] + 1e-15)


def test_width_scales_quadratically(quad):
    """The remainder is second order: width(rho)/rho^2 tends to a constant as rho -> 0."""
    w, dyn = quad
    a = w.nominal()[5].astype(np.float64)
    base = w.radii[5].astype(np.float64)
    ratios = []
    for s in (1e-1, 1e-2, 1e-3):
        lo, hi = a - s * base, a + s * base
        Rl, Rh = pbh.pbh(dyn, a, lo, hi)
        ratios.append((Rh[3] - Rl[3]) / s ** 2)
    assert abs(ratios[1] / ratios[2] - 1) < 0.02 and abs(ratios[0] / ratios[2] - 1) < 0.2


def test_chain_decomposes_per_quadrotor():
    """Springs are linear: each quadrotor's rows of the chain equal the single-quadrotor bound."""
    w = inputs.quad_chain(n_traj=2, horizon=4, with_G=True)
    chain = dynamics.QuadChain(28, **w.params, spring_k=0.5)
    single = dynamics.QuadChain(1, **w.params)
    t = 3
    a = w.nominal()[t].astype(np.float64)
    lo, hi = pbh.box_from_set(a, G=w.G[t])
    Rl, Rh = pbh.pbh(chain, a, lo, hi)
    for i in (0, 13, 27):
        idx = [chain.ix(i, s) for s in range(6)] + [chain.iu(i, 0), chain.iu(i, 1)]
        sl, sh = pbh.pbh(single, a[idx], lo[idx], hi[idx])
        assert np.allclose(Rl[6 * i:6 * i + 6], sl, rtol=0, atol=1e-15)
        assert np.allclose(Rh[6 * i:6 * i + 6], sh, rtol=0, atol=1e-15)


def test_zonotope_hull_and_soundness():
    """Eq. 21 hull: every zonotope point lies in c +- ||G||_{1,r}; the bound contains sampled remainders."""
    w = inputs.quad_chain(n_traj=1, horizon=3, n_quads=3, with_G=True)
    dyn = dynamics.QuadChain(3, **w.params, spring_k=0.5)
    rng = np.random.default_rng(4)
    for t in range(3):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, G=w.G[t])
        P = sampling.zonotope_points(a, w.G[t], 20000, rng)
        assert np.all(P >= lo - 1e-12) and np.all(P <= hi + 1e-12)
        ext = np.argmax(P[:, 2])     # a sign vertex attains the hull on that row
        assert P[ext, 2] >= hi[2] - 1e-9
        Rl, Rh = pbh.pbh(dyn, a, lo, hi)
        R = sampling.remainders(dyn.f_batch, a, dyn.jacobian(a), np.concatenate(
            [P, sampling.box_points(lo, hi, 20000, rng)]))
        assert np.all(R >= Rl - 1e-12) and np.all(R <= Rh + 1e-12)


def test_interval_trig_exact_ranges():
    """Interval sin/cos against dense evaluation (their extremes are the textbook critical points)."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        lo = rng.uniform(-20, 20)
        hi = lo + rng.uniform(0, 7)
        xs = np.linspace(lo, hi, 20001)
        s = dynamics.iv_sin(lo, hi)
        c = dynamics.iv_cos(lo, hi)
        assert s[0] <= np.sin(xs).min() + 1e-12 and s[1] >= np.sin(xs).max() - 1e-12
        assert c[0] <= np.cos(xs).min() + 1e-12 and c[1] >= np.cos(xs).max() - 1e-12
        assert s[1] - s[0] <= np.sin(xs).max() - np.sin(xs).min() + 1e-6
        assert c[1] - c[0] <= np.cos(xs).max() - np.cos(xs).min() + 1e-6


def test_nominal_outside_set_is_hulled():
    """Thm. 1 needs alpha~ in X: a set that misses the nominal is hulled with it."""
    a = np.array([0.0, 1.0, 2.0])
    lo, hi = pbh.box_from_set(a, radii=np.array([0.1, 0.1, 0.1]), center=np.array([0.5, 1.0, 1.0]))
    assert lo[0] == 0.0 and hi[0] == pytest.approx(0.6) and hi[2] == 2.0 and lo[2] == pytest.approx(0.9)


def test_gamma_map():
    c, rad = pbh.gamma_map(np.array([-1.0, 0.0]), np.array([3.0, 0.0]), pad=1e-6)
    assert c.tolist() == [1.0, 0.0] and rad.tolist() == [2.0 + 1e-6, 1e-6]


def test_partitioned_pbh_is_inside_plain_and_contains_the_exact_range():
    """Input-domain partitioning at the nominal: every piece's Thm. 1 bound is an interval extension over
    a subset of the box, so the hull of the pieces lies inside the plain bound (inclusion monotonicity),
    and it still contains the exact range (1-D analysis of the planar quadrotor)."""
    from oracle import exact
    w = inputs.planar_quad()
    dyn = dynamics.QuadChain(1, **w.params)
    gain = []
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        P = pbh.pbh(dyn, a, lo, hi)
        S = pbh.pbh_partitioned(dyn, a, lo, hi, dims=[2, 6, 7])
        assert np.all(S[0] >= P[0] - 1e-15) and np.all(S[1] <= P[1] + 1e-15)
        el, eh = exact.quad_exact_range(dyn, a, lo, hi)
        assert np.all(S[0] <= el + 1e-12) and np.all(S[1] >= eh - 1e-12)
        gain.append((S[1] - S[0]).sum() / (P[1] - P[0]).sum())
    # the pieces keep the nominal, so every |Delta_j| keeps its range: the gain is small (0.998 here)
    assert np.mean(gain) <= 1.0


def test_partition_pieces_cover_the_box():
    rng = np.random.default_rng(80)
    a = rng.normal(size=5)
    lo, hi = a - rng.uniform(0.1, 1.0, 5), a + rng.uniform(0.1, 1.0, 5)
    pieces = list(pbh.split_pieces(a, lo, hi, [0, 3]))
    assert len(pieces) == 4
    for lp, hp in pieces:   # every piece contains the nominal and lies in the box
        assert np.all(lp <= a) and np.all(a <= hp) and np.all(lp >= lo) and np.all(hp <= hi)
    X = lo + rng.uniform(0, 1, (1000, 5)) * (hi - lo)
    inside = np.zeros(len(X), bool)
    for lp, hp in pieces:
        inside |= np.all((X >= lp) & (X <= hp), axis=1)
    assert inside.all()


def test_path_orderings():
    """Thm. 1 holds for any path order (the proof only needs a coordinate-wise path): every order's bound
    contains the exact range of the planar quadrotor; the identity permutation is the default; for the
    satellite (constant Hessian) every order gives the same, exact, bound."""
    from oracle import dynamics3d, exact
    rng = np.random.default_rng(81)
    w = inputs.planar_quad()
    dyn = dynamics.QuadChain(1, **w.params)
    orders = [list(range(8)), [6, 7, 0, 1, 2, 3, 4, 5], list(range(8))[::-1]] + \
        [list(rng.permutation(8)) for _ in range(3)]
    for t in range(0, w.T, 4):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        el, eh = exact.quad_exact_range(dyn, a, lo, hi)
        base = pbh.pbh(dyn, a, lo, hi)
        for od in orders:
            l, h = pbh.pbh(dyn, a, lo, hi, order=od)
            assert np.all(l <= el + 1e-12) and np.all(h >= eh - 1e-12)
        l0, h0 = pbh.pbh(dyn, a, lo, hi, order=list(range(8)))
        assert np.array_equal(l0, base[0]) and np.array_equal(h0, base[1])
    sat = dynamics3d.Satellite()
    a = np.concatenate([rng.normal(size=4) / 2, rng.uniform(-1, 1, 6)])
    lo, hi = a - 0.1, a + 0.1
    b = pbh.pbh(sat, a, lo, hi)
    for _ in range(4):
        l, h = pbh.pbh(sat, a, lo, hi, order=list(rng.permutation(10)))
        assert np.allclose(l, b[0], rtol=1e-13, atol=1e-16) and np.allclose(h, b[1], rtol=1e-13, atol=1e-16)


def test_recentred_partition_contains_exact_range_and_converges():
    """Re-centred input-domain partitioning of the attitude: K = 1 on a box centred at the nominal is the
    plain bound (beta = nominal); for K = 2, 4, 16 every bound contains the exact range (1-D analysis of the
    planar quadrotor, w.r.t. the same A); the width decreases with K and the excess over the exact range
    shrinks at least fourfold from K = 1 to K = 16 (it vanishes as the pieces shrink)."""
    from oracle import exact
    w = inputs.planar_quad()
    dyn = dynamics.QuadChain(1, **w.params)
    ex1, ex16 = [], []
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, radii=w.radii[t])
        P = pbh.pbh(dyn, a, lo, hi)
        R1 = pbh.pbh_recentred(dyn, a, lo, hi, [2], 1)   # beta = the FP32 midpoint: the nominal up to an ulp
        tol = 1e-6 * (P[1] - P[0]).max()
        assert np.allclose(R1[0], P[0], rtol=0, atol=tol) and np.allclose(R1[1], P[1], rtol=0, atol=tol)
        el, eh = exact.quad_exact_range(dyn, a, lo, hi)
        widths = []
        for K in (2, 4, 16):
            l, h = pbh.pbh_recentred(dyn, a, lo, hi, [2], K)
            assert np.all(l <= el + 1e-12) and np.all(h >= eh - 1e-12), (t, K)
            widths.append((h - l).sum())
            if K == 16:
                ex16.append((h - l).sum() - (eh - el).sum())
        assert widths[0] >= widths[1] >= widths[2]
        ex1.append((P[1] - P[0]).sum() - (eh - el).sum())
    assert np.sum(ex16) <= 0.25 * np.sum(ex1), (np.sum(ex16), np.sum(ex1))


def test_recentred_partition_sampled_on_the_chain():
    """Two coupled quadrotors with zonotope hulls, every attitude cut into 8 re-centred pieces: the bound
    (each row from its own quadrotor's attitude pieces) contains sampled remainders."""
    from oracle import sampling
    w = inputs.quad_chain(n_traj=1, horizon=3, n_quads=2)
    dyn = dynamics.QuadChain(2, **w.params, spring_k=w.spring_k)
    rng = np.random.default_rng(81)
    for t in range(w.T):
        a = w.nominal()[t].astype(np.float64)
        lo, hi = pbh.box_from_set(a, G=w.G[t])
        l, h = pbh.pbh_recentred(dyn, a, lo, hi, [dyn.ix(0, 2), dyn.ix(1, 2)], 8)
        P = sampling.box_points(lo, hi, 20000, rng)
        R = sampling.remainders(lambda X: np.array([dyn.f(x) for x in X]), a, dyn.jacobian(a), P)
        assert np.all(R >= l - 1e-12) and np.all(R <= h + 1e-12)
