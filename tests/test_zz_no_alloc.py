"""The allocation-free time average (arp_coarse_avg_static) against the
context-based arp_coarse_avg, on two calls in a row.

arp_coarse_avg_static serves callers that cannot call cudaMalloc (a framework
with a fixed device-memory budget, a latency-critical loop that cannot afford
the allocation's synchronisation): it keeps its tables and workspaces in one
16 MiB static device array instead of a context.  This file is collected last
so that a run stopping at the first failure has already run every other test;
it also passes on its own in a fresh process."""
import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _reference(b, n, eps, dT, m, x):
    torch = cuda_or_skip()
    with b.Solver(n, eps, 1e-4, x.shape[0], dT, dT / 8, m) as s:
        xin = to_dev(x)
        out = torch.empty_like(xin)
        b.arp_coarse_avg(s.ctx, xin, out)
        return to_host(out)


def test_static_time_average_matches_context_path_on_two_calls():
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    cases = [(64, 1e-2, 0.0625, 32, ri.random_batch(64, 8, 16.0, 5, 300) * 64.0),
             (512, 1e-3, 10 / 256, 64, ri.random_batch(512, 32, 256.0, 3, 400) * 512.0)]
    for n, eps, dT, m, x in cases:   # two calls in a row, different sizes
        xin = to_dev(x)
        out = torch.full_like(xin, float("nan"))
        b.arp_coarse_avg_static(n, eps, dT, m, xin, out)
        got = to_host(out)
        ref = _reference(b, n, eps, dT, m, x)
        assert np.all(np.isfinite(got))
        assert per_state_rel_l2(got, ref).max() <= TOL64


def test_static_time_average_rejects_sizes_beyond_its_array():
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    n = 2048
    x = torch.zeros((1, 3, n // 2 + 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(b.ArpError) as ei:
        b.arp_coarse_avg_static(n, 1e-3, 0.01, 4096, x, torch.empty_like(x))
    assert ei.value.status == b.ARP_EINVAL


def test_static_time_average_several_passes_against_oracle():
    # 40 states at N = 512, M = 64: more than one pass through the array holds
    # (29 states), so the batch runs in two passes.  Checked against the
    # context path and directly against the oracle's time average (Eq. 2.1,
    # Algorithm 1).
    torch = cuda_or_skip()
    from oracle import rsw as o
    from paper_1303_6615_gb300 import binding as b
    n, eps, dT, m = 512, 1e-3, 10 / 256, 64
    x = ri.random_batch(n, 32, 256.0, 40, 500) * 512.0
    xin = to_dev(x)
    out = torch.full_like(xin, float("nan"))
    b.arp_coarse_avg_static(n, eps, dT, m, xin, out)
    got = to_host(out)
    assert np.all(np.isfinite(got))
    assert per_state_rel_l2(got, _reference(b, n, eps, dT, m, x)).max() <= TOL64
    p = o.Params(n, eps, 1e-4, dT, dT / 8, m)
    assert per_state_rel_l2(got, o.nbar(x, p)).max() <= TOL64
