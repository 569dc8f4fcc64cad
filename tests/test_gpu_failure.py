"""Failure detection without a GPU fault: a bounded device wait that nothing ends reports a status and
returns (the context stays usable); non-finite inputs and bad arguments are caught as statuses."""
import numpy as np
import pytest
import torch

from paper_2607_01203_b300 import binding, inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports():
    lib = binding.lib()
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    waited = torch.zeros(1, dtype=torch.int64, device="cuda")
    limit = 50_000_000   # 50 ms
    binding.check(lib.leb_selftest_wait_timeout(flags.data_ptr(), limit, waited.data_ptr(), None), "wait")
    torch.cuda.synchronize()
    assert int(flags.item()) == binding.ASYNC_TIMEOUT
    assert limit <= int(waited.item()) < limit + 1_000_000_000
    # the context is still usable: a normal bounds call right after
    w = inputs.planar_quad()
    h = binding.quad_chain(1, **w.params)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    out = h.bounds(t(w.x_nom), t(w.u_nom), radii=t(w.radii))
    torch.cuda.synchronize()
    assert int(out["flags"].item()) == 0 and torch.all(torch.isfinite(out["r_lo"]))
    assert lib.leb_selftest_wait_timeout(None, limit, waited.data_ptr(), None) == binding.LEB_ERR_INVALID_ARG


def test_zonotope_pbh_kernel_returns_when_its_waits_run_out():
    """The zonotope PBH kernel with a 1 microsecond limit on its pipeline waits (producer, consumers,
    writer): waits run out while the pipeline still runs, in whichever warp. Every warp must leave (the
    consumers' barriers are bounded too), the call must return with LEB_ASYNC_TIMEOUT or, if no wait ran
    out, complete bounds; the next call with the library's limit gives the bits of a clean call."""
    lib = binding.lib()
    w = inputs.quad_chain(n_traj=8, horizon=50)
    h = binding.quad_chain(28, **w.params, spring_k=w.spring_k)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    x, u, G = t(w.x_nom), t(w.u_nom), t(w.G)
    ref = h.bounds(x, u, G=G)
    torch.cuda.synchronize()
    assert int(ref["flags"].item()) == 0
    ref = {k: v.clone() for k, v in ref.items()}
    timeouts = 0
    try:
        binding.check(lib.leb_selftest_set_wait_limit(h.h, 1000), "set_wait_limit")
        for _ in range(5):
            out = h.bounds(x, u, G=G)
            torch.cuda.synchronize()
            f = int(out["flags"].item())
            assert f in (0, binding.ASYNC_TIMEOUT), f
            timeouts += f == binding.ASYNC_TIMEOUT
            if f == 0:
                assert torch.equal(out["r_lo"], ref["r_lo"]) and torch.equal(out["r_hi"], ref["r_hi"])
    finally:
        binding.check(lib.leb_selftest_set_wait_limit(h.h, 0), "set_wait_limit")
    assert timeouts > 0
    out = h.bounds(x, u, G=G)
    torch.cuda.synchronize()
    assert int(out["flags"].item()) == 0
    for k in ("r_lo", "r_hi", "A", "B"):
        assert torch.equal(out[k], ref[k]), k
    assert lib.leb_selftest_set_wait_limit(None, 0) == binding.LEB_ERR_INVALID_ARG
