"""leb_bounds_static (no workspace argument, library-owned scratch) against leb_bounds.

Callers such as a control loop whose device memory is fixed after start-up cannot hand the library a
workspace; this entry point serves them from a static scratch array. Both entry points launch the same
bound kernel, so the results must agree within the tolerance of the PBH tests — here they are compared
for equality — on two calls in a row (the second call reuses the scratch left by the first).
Collected last so that a failure here does not stop the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2607_01203_b300 import binding, inputs

pytestmark = pytest.mark.gpu


def _t(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to("cuda", dtype)


def _static(h, x, u, sd, bd, T, n_rows, nA, nB):
    f32 = dict(device="cuda", dtype=torch.float32)
    lo, hi = torch.empty(n_rows, **f32), torch.empty(n_rows, **f32)
    A, B = torch.empty(nA, **f32), torch.empty(nB, **f32)
    flags = torch.zeros(1, device="cuda", dtype=torch.int32)
    st = binding.lib().leb_bounds_static(h.h, None if bd is None else C.byref(bd), T, C.c_void_p(x.data_ptr()),
                                         C.c_void_p(u.data_ptr()), C.byref(sd), C.c_void_p(lo.data_ptr()),
                                         C.c_void_p(hi.data_ptr()), C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                                         C.c_void_p(flags.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    binding.check(st, "leb_bounds_static")
    torch.cuda.synchronize()
    return lo, hi, A, B, flags


def test_static_matches_workspace_entry_point_twice():
    w = inputs.quad_chain(n_traj=3, horizon=(2, 6), n_quads=28)
    h = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
    x, u, G = _t(w.x_nom), _t(w.u_nom), _t(w.G)
    ref = h.bounds(x, u, G=G)
    torch.cuda.synchronize()
    sd = binding.Handle.set_desc(G=G)
    for _ in range(2):
        lo, hi, A, B, flags = _static(h, x, u, sd, None, w.T, w.T * 168, w.T * 168 * 168, w.T * 168 * 56)
        assert flags.item() == 0
        assert torch.equal(lo.view(w.T, 168), ref["r_lo"]) and torch.equal(hi.view(w.T, 168), ref["r_hi"])
        assert torch.equal(A.view_as(ref["A"]), ref["A"]) and torch.equal(B.view_as(ref["B"]), ref["B"])


def test_static_uneven_batch_and_size_limit():
    nqs, horizons = [28, 3, 9], [3, 4, 2]
    parts = [inputs.quad_chain(seed=5000 + i, n_traj=1, horizon=hz, n_quads=nq) for i, (nq, hz) in
             enumerate(zip(nqs, horizons))]
    X = _t(np.concatenate([p.x_nom.reshape(-1) for p in parts]))
    U = _t(np.concatenate([p.u_nom.reshape(-1) for p in parts]))
    G = _t(np.concatenate([p.G.reshape(-1) for p in parts]))
    offs = _t(np.concatenate([[0], np.cumsum(horizons)]).astype(np.int32), torch.int32)
    nq_t = _t(np.array(nqs, np.int32), torch.int32)
    h = binding.quad_chain(28, **parts[0].params, spring_k=0.5)
    ref = h.bounds(X, U, G=G, traj_offsets=offs, traj_nquads=nq_t, n_gen_per_quad=12)
    torch.cuda.synchronize()
    sd = binding.SetDesc(binding.SET_ZONO, None, None, C.c_void_p(G.data_ptr()), 12)
    bd = binding.BatchDesc(3, C.c_void_p(offs.data_ptr()), C.c_void_p(nq_t.data_ptr()))
    T = int(sum(horizons))
    rows = sum(6 * q * hz for q, hz in zip(nqs, horizons))
    nA = sum(36 * q * q * hz for q, hz in zip(nqs, horizons))
    nB = sum(12 * q * q * hz for q, hz in zip(nqs, horizons))
    for _ in range(2):
        lo, hi, A, B, flags = _static(h, X, U, sd, bd, T, rows, nA, nB)
        assert torch.equal(lo, ref["r_lo"]) and torch.equal(hi, ref["r_hi"]) and torch.equal(A, ref["A"])
    big = binding.BatchDesc(binding.lib().leb_bounds_static_max_traj() + 1, C.c_void_p(offs.data_ptr()),
                            C.c_void_p(nq_t.data_ptr()))
    flags = torch.zeros(1, device="cuda", dtype=torch.int32)
    st = binding.lib().leb_bounds_static(h.h, C.byref(big), T, C.c_void_p(X.data_ptr()), C.c_void_p(U.data_ptr()),
                                         C.byref(sd), C.c_void_p(lo.data_ptr()), C.c_void_p(hi.data_ptr()), None, None,
                                         C.c_void_p(flags.data_ptr()), None)
    assert st == -3  # LEB_ERR_WORKSPACE: more trajectories than the fixed scratch holds
