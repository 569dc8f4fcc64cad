"""GPU parity of the tube centre and width after the LEB (Sec. V-A, Eqs. 18b, 20-21) against the FP64
oracle, through the C ABI.

Tolerance (from the kernel's FP32 arithmetic): sigma is a sum of m = k n_x non-negative products per
block row, every product and sum rounded up, so it exceeds the exact value by at most about
m 2^-23 of the sum; mu is the midpoint of a directed-rounding enclosure of the same length. Per row:
  * containment: [mu_g - sigma_g, mu_g + sigma_g] contains [mu_o - sigma_o, mu_o + sigma_o] (up to FP64
    noise, 1e-12 of the scale);
  * width: sigma_g <= sigma_o + |mu_g - mu_o| + m 2^-22 (sigma_o + sum_j |Phi_{k,j}| |c_j|).
"""
import numpy as np
import pytest
import torch

from oracle import tube as otube
from paper_2607_01203_b300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV, torch.float32)


def run(w, e=None):
    e = w.e if e is None else e
    mu, sigma, fl = binding.tube(_t(w.Phi), _t(e), _t(w.c), _t(w.r), w.n_traj, w.N, w.n_x, w.n_u)
    torch.cuda.synchronize()
    return mu.cpu().numpy().astype(np.float64), sigma.cpu().numpy().astype(np.float64), int(fl.item())


def check(w, mu, sigma, b, ks=None, e=None):
    e = w.e if e is None else e
    sl = slice(b * w.N, (b + 1) * w.N)
    E = e.astype(np.float64) if e.ndim == 1 else [v for v in e[sl].astype(np.float64)]
    Phi = w.Phi[b].astype(np.float64)
    c, r = w.c[sl].astype(np.float64), w.r[sl].astype(np.float64)
    mo, so = otube.tube(Phi, w.N, c, r, E)
    for k in (range(w.N + 1) if ks is None else ks):
        scale = np.abs(mo[k]) + so[k] + 1e-300
        assert np.all(mu[b, k] - sigma[b, k] <= mo[k] - so[k] + 1e-12 * scale), (b, k)
        assert np.all(mu[b, k] + sigma[b, k] >= mo[k] + so[k] - 1e-12 * scale), (b, k)
        if k == 0:
            assert np.all(mu[b, 0] == 0) and np.all(sigma[b, 0] == 0)
            continue
        m = k * w.n_x
        absc = sum(np.abs(Phi[otube.block_index(k, j)]) @ np.abs(c[j]) for j in range(k))
        tol = so[k] + np.abs(mu[b, k] - mo[k]) + m * 2.0 ** -22 * (so[k] + absc)
        assert np.all(sigma[b, k] <= tol), (b, k, np.max(sigma[b, k] - tol))


@pytest.mark.parametrize("n_x,n_u,N,n_traj", [(12, 4, 25, 3), (7, 3, 10, 2), (2, 1, 1, 4)])
def test_parity_every_timestep(n_x, n_u, N, n_traj):
    w = inputs.tube(n_traj=n_traj, N=N, n_x=n_x, n_u=n_u, keep_model=False)
    mu, sigma, fl = run(w)
    assert fl == 0
    for b in range(n_traj):
        check(w, mu, sigma, b)


def test_per_timestep_disturbance_scaling():
    w = inputs.tube(n_traj=2, N=9, n_x=8, n_u=2, keep_model=False)
    e = (np.random.default_rng(72).uniform(-5e-3, 5e-3, (w.n_traj * w.N, w.n_x))).astype(np.float32)
    mu, sigma, fl = run(w, e)
    assert fl == 0
    for b in range(w.n_traj):
        check(w, mu, sigma, b, e=e)


def test_168_state_shape_sampled():
    """The paper's 168-state coupled system shape (n_x = 168, n_u = 56, horizon 25), 4 trajectories in one
    launch; sampled (trajectory, k) against the oracle."""
    w = inputs.tube(n_traj=4, N=25, n_x=168, n_u=56, keep_model=False)
    mu, sigma, fl = run(w)
    assert fl == 0
    check(w, mu, sigma, 0, ks=[0, 1, 2, 13, 25])
    check(w, mu, sigma, 3, ks=[1, 24, 25])


def test_edge_cases():
    w = inputs.tube(n_traj=2, N=5, n_x=4, n_u=1, keep_model=False)
    # no trajectories / horizon 0
    fl = torch.ones(1, dtype=torch.int32, device=DEV)
    binding.check(binding.lib().leb_tube(0, 5, 4, 1, None, None, 0, None, None, None, None, fl.data_ptr(), None),
                  "leb_tube")
    torch.cuda.synchronize()
    assert int(fl.item()) == 0
    mu = torch.ones(3, 1, 5, device=DEV)
    sg = torch.ones(3, 1, 5, device=DEV)
    binding.check(binding.lib().leb_tube(3, 0, 4, 1, None, None, 0, None, None, mu.data_ptr(), sg.data_ptr(),
                                         fl.data_ptr(), None), "leb_tube")
    torch.cuda.synchronize()
    assert torch.all(mu == 0) and torch.all(sg == 0)
    # a non-finite response poisons only the rows that read it
    Phi = w.Phi.copy()
    Phi[1, otube.block_index(3, 1), 2, 0] = np.inf
    w2 = inputs.TubeWorkload(w.n_traj, w.N, w.n_x, w.n_u, Phi, w.c, w.r, w.e, None, None, None)
    mu, sigma, fl = run(w2)
    assert fl & 1
    assert sigma[1, 3, 2] == np.inf and mu[1, 3, 2] == 0
    bad = np.zeros_like(sigma, dtype=bool)
    bad[1, 3, 2] = True
    assert np.all(np.isfinite(sigma[~bad]))
    check(w, mu, sigma, 0)
    # an oversized shared-memory request is refused on the host before anything is launched
    small = torch.zeros(16, device=DEV)
    flg = torch.zeros(1, dtype=torch.int32, device=DEV)
    st = binding.lib().leb_tube(1, 4000, 168, 0, small.data_ptr(), small.data_ptr(), 0, small.data_ptr(),
                                small.data_ptr(), small.data_ptr(), small.data_ptr(), flg.data_ptr(), None)
    assert st == binding.LEB_ERR_UNSUPPORTED
