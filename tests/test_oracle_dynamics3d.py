"""Pins of the oracle's satellite and 3-D quadrotor models (App. A) and of Thm. 1 on them (CPU only)."""
import itertools

import numpy as np
import pytest

from oracle import dynamics3d, pbh, sampling


def _sat_point(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    return np.concatenate([q, rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)])


def _quad_point(rng, nq=1):
    a = []
    for _ in range(nq):
        a.append(np.concatenate([rng.uniform(-1, 1, 3), rng.uniform(-0.5, 0.5, 2), rng.uniform(-np.pi, np.pi, 1),
                                 rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)]))
    u = [np.concatenate([rng.uniform(5, 15, 1), rng.uniform(-0.1, 0.1, 3)]) for _ in range(nq)]
    return np.concatenate(a + u)


def test_jacobian_matches_finite_differences():
    rng = np.random.default_rng(50)
    for d, pt in ((dynamics3d.Satellite(), _sat_point), (dynamics3d.Quad3D(1), _quad_point),
                  (dynamics3d.Quad3D(3, coup_alpha=0.75, coup_gamma=0.25), lambda r: _quad_point(r, 3))):
        for _ in range(3):
            a = pt(rng)
            J = d.jacobian(a)
            Jfd = np.zeros_like(J)
            for i in range(d.n):
                e = np.zeros(d.n)
                e[i] = 1e-6
                Jfd[:, i] = (d.f(a + e) - d.f(a - e)) / 2e-6
            assert np.abs(J - Jfd).max() < 1e-7


def test_hessian_table_matches_automatic_differentiation():
    """Every hand-derived entry (and the absence of all others) against autograd second derivatives."""
    rng = np.random.default_rng(51)
    for d, pt in ((dynamics3d.Satellite(), _sat_point), (dynamics3d.Quad3D(1), _quad_point),
                  (dynamics3d.Quad3D(2, coup_alpha=0.75, coup_gamma=0.25), lambda r: _quad_point(r, 2))):
        for _ in range(4):
            a = pt(rng)
            assert np.abs(d.hessian_point(a) - d.hessian_autodiff(a)).max() < 1e-12


def test_satellite_bound_is_the_exact_range():
    """The satellite model is bilinear and every row's terms involve disjoint coordinate pairs, so the
    remainder is multilinear on the box (extremes at vertices) and Thm. 1's term-wise sum is exact."""
    d = dynamics3d.Satellite()
    rng = np.random.default_rng(52)
    V = np.array(list(itertools.product((0.0, 1.0), repeat=d.n)))
    for eps in (0.01, 0.1, 0.2):
        a = _sat_point(rng)
        lo, hi = a - eps, a + eps
        Rl, Rh = pbh.pbh(d, a, lo, hi)
        R = sampling.remainders(d.f_batch, a, d.jacobian(a), lo + V * (hi - lo))
        assert np.allclose(Rl, R.min(0), rtol=1e-10, atol=1e-14) and np.allclose(Rh, R.max(0), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("nq,coup", [(1, 0.0), (3, 1.0)])
def test_quad3d_bound_contains_sampled_remainders(nq, coup):
    d = dynamics3d.Quad3D(nq, coup_alpha=0.75 * coup, coup_gamma=0.25 * coup)
    rng = np.random.default_rng(53 + nq)
    for eps in (0.01, 0.05, 0.2):
        a = _quad_point(rng, nq)
        lo, hi = a - eps, a + eps
        Rl, Rh = pbh.pbh(d, a, lo, hi)
        R = sampling.remainders(d.f_batch, a, d.jacobian(a), sampling.box_points(lo, hi, 20000, rng))
        # FP64 evaluation of f(alpha) - f(alpha~) - J delta carries rounding noise of ~1e-16 (the linear rows'
        # remainder is exactly 0)
        scale = np.maximum(np.abs(Rl), np.abs(Rh)) + 1e-14
        assert np.all(R.min(0) >= Rl - 1e-12 * scale - 1e-14) and np.all(R.max(0) <= Rh + 1e-12 * scale + 1e-14)
        # the linear rows (positions, and the body rates through their bilinear term only) stay small
        assert np.all(Rh - Rl >= 0)


def test_quad3d_corollary1_and_quadratic_scaling():
    d = dynamics3d.Quad3D(1)
    rng = np.random.default_rng(55)
    for _ in range(10):
        a = _quad_point(rng)
        rad = rng.uniform(0.01, 0.2, d.n)
        lo, hi = a - rad, a + rad
        P = pbh.pbh(d, a, lo, hi)
        E = pbh.ih_expand(d, a, lo, hi)
        C = pbh.ih_classic(d, a, lo, hi)
        assert np.all(E[0] <= P[0] + 1e-14) and np.all(P[1] <= E[1] + 1e-14)
        assert np.all(C[0] <= E[0] + 1e-14) and np.all(E[1] <= C[1] + 1e-14)
    a = _quad_point(rng)
    base = rng.uniform(0.5, 1.0, d.n)
    w = []
    for s in (1e-2, 1e-3, 1e-4):
        Rl, Rh = pbh.pbh(d, a, a - s * base, a + s * base)
        w.append((Rh - Rl).sum() / s ** 2)
    assert abs(w[1] / w[2] - 1) < 0.02 and abs(w[0] / w[2] - 1) < 0.2
