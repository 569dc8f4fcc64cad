"""Pins of the FP64 gradient oracle of the PBH bound (Thm. 1, differentiable LEBs of Sec. IV-D), CPU only."""
import math

import numpy as np
import pytest
import torch

from oracle import dynamics, pbh, pbh_grad
from paper_2607_01203_b300 import inputs


@pytest.fixture(scope="module")
def quad():
    w = inputs.planar_quad()
    return w, dynamics.QuadChain(1, **w.params)


def _np_bound(dyn, a, r):
    lo, hi = pbh.box_from_set(a, radii=r)
    return pbh.pbh(dyn, a, lo, hi)


def _points(dyn, rng, n):
    for _ in range(n):
        a = rng.normal(size=dyn.n)
        a[dyn.n_x:] = rng.uniform(3.0, 7.0, size=dyn.n_u)          # thrusts as in the workloads
        r = rng.uniform(0.01, 0.1, size=dyn.n)
        yield a, r


def test_values_match_numpy_oracle(quad):
    """The torch evaluation of Thm. 1 is the NumPy one (oracle.pbh), term for term."""
    w, dyn = quad
    chain = dynamics.QuadChain(4, **w.params, spring_k=0.5)
    rng = np.random.default_rng(20)
    for d in (dyn, chain):
        for a, r in _points(d, rng, 6):
            lo_t, hi_t = pbh_grad.pbh_torch(d, torch.tensor(a), torch.tensor(r))
            lo_n, hi_n = _np_bound(d, a, r)
            assert np.allclose(lo_t.numpy(), lo_n, rtol=1e-13, atol=1e-16)
            assert np.allclose(hi_t.numpy(), hi_n, rtol=1e-13, atol=1e-16)


def test_gradient_matches_central_differences(quad):
    """VJP vs central differences (h = 1e-6) of the independent NumPy bound, random cotangents."""
    w, dyn = quad
    chain = dynamics.QuadChain(3, **w.params, spring_k=0.5)
    rng = np.random.default_rng(21)
    h = 1e-6
    for d in (dyn, chain):
        for a, r in _points(d, rng, 4):
            g_lo, g_hi = rng.normal(size=d.n_x), rng.normal(size=d.n_x)
            gx, gu, gr = pbh_grad.pbh_vjp(d, a, r, g_lo, g_hi)
            ga = np.concatenate([gx, gu])

            def L(a_, r_):
                lo_, hi_ = _np_bound(d, a_, r_)
                return float(g_lo @ lo_ + g_hi @ hi_)

            fa = np.zeros(d.n)
            fr = np.zeros(d.n)
            for i in range(d.n):
                e = np.zeros(d.n)
                e[i] = h
                fa[i] = (L(a + e, r) - L(a - e, r)) / (2 * h)
                fr[i] = (L(a, r + e) - L(a, r - e)) / (2 * h)
            scale = np.abs(fa).max() + np.abs(fr).max()
            assert np.abs(ga - fa).max() <= 1e-6 * scale
            assert np.abs(gr - fr).max() <= 1e-6 * scale


def test_closed_form_at_level_attitude(quad):
    """phi~ = 0: the v_x row's upper bound is 1/2 c S sin(rho) rho^2 + c rho (rho_1 + rho_2) (c = dt/m;
    [sin] over [-rho, rho] tops at sin(rho), [cos] tops at the interior maximum 1), so its gradient is
    known in closed form; the v_y row's lower bound -1/2 c S rho^2 - c sin(rho) rho (rho_1 + rho_2) has
    known radius derivatives."""
    w, dyn = quad
    c = dyn.dt / dyn.m
    a = np.zeros(dyn.n)
    a[6], a[7] = 4.0, 5.5
    r = np.zeros(dyn.n)
    rho, r1, r2 = 0.07, 0.03, 0.05
    r[2], r[6], r[7] = rho, r1, r2
    S = a[6] + a[7]
    g_hi = np.zeros(dyn.n_x)
    g_hi[3] = 1.0
    gx, gu, gr = pbh_grad.pbh_vjp(dyn, a, r, np.zeros(dyn.n_x), g_hi)
    assert math.isclose(gx[2], 0.5 * c * S * math.cos(rho) * rho * rho, rel_tol=1e-12)
    assert math.isclose(gu[0], 0.5 * c * math.sin(rho) * rho * rho, rel_tol=1e-12)
    assert math.isclose(gu[1], gu[0], rel_tol=1e-12)
    assert math.isclose(gr[2], 0.5 * c * S * (math.cos(rho) * rho * rho + 2 * rho * math.sin(rho)) + c * (r1 + r2),
                        rel_tol=1e-12)
    assert math.isclose(gr[6], c * rho, rel_tol=1e-12) and math.isclose(gr[7], c * rho, rel_tol=1e-12)
    g_lo = np.zeros(dyn.n_x)
    g_lo[4] = 1.0
    _, gu, gr = pbh_grad.pbh_vjp(dyn, a, r, g_lo, np.zeros(dyn.n_x))
    assert math.isclose(gu[0], -0.5 * c * rho * rho, rel_tol=1e-12)
    assert math.isclose(gr[2], -c * S * rho - c * (math.cos(rho) * rho + math.sin(rho)) * (r1 + r2), rel_tol=1e-12)
    assert math.isclose(gr[6], -c * math.sin(rho) * rho, rel_tol=1e-12)


def test_linear_rows_and_other_coordinates_have_zero_gradient(quad):
    """Only the v_x, v_y rows are curved and they depend on (phi, u_1, u_2) alone (Hessian table)."""
    w, dyn = quad
    chain = dynamics.QuadChain(3, **w.params, spring_k=0.5)
    rng = np.random.default_rng(22)
    for a, r in _points(chain, rng, 3):
        gx, gu, gr = pbh_grad.pbh_vjp(chain, a, r, rng.normal(size=chain.n_x), rng.normal(size=chain.n_x))
        for i in range(chain.nq):
            for s in (0, 1, 3, 4, 5):
                assert gx[chain.ix(i, s)] == 0.0 and gr[chain.ix(i, s)] == 0.0
