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
