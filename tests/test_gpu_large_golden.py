"""Full-width parity of the single large workload (N = 512, 256 slices, M = 64):
the coarse predictor U^0 and the first iterate U^1 on every slice, against the
FP64 oracle's values stored in tests/golden/rsw-N512-S256-M64_k01.npz (written
by tests/golden/make_large_golden.py, which calls only the oracle).

The FP32-bulk solve is called exactly as the bench calls it: arp_set_initial,
then arp_parareal_solve (pipelined across iterations where the device allows),
with K_max = 0 for the predictor and K_max = 1 for the first iterate.  Bar:
relative L2 per slice <= 1e-5 (FP32 bulk) and <= 1e-10 (the FP64 path)."""
import os

import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rsw-N512-S256-M64_k01.npz")
TOL = {0: 1e-10, 1: 1e-5}


def _golden():
    g = np.load(GOLDEN)
    w = ri.LARGE_N512
    assert str(g["workload"]) == w.name
    H = w.n_grid // 2 + 1
    K = int(g["kept"])
    out = []
    for key in ("U0", "U1"):
        U = np.zeros((w.slices + 1, 3, H), dtype=np.complex128)
        U[..., :K + 1] = g[key]
        out.append(U)
    return out, float(g["change1"])


@pytest.mark.parametrize("precision", [1, 0], ids=["fp32-solve", "fp64-solve"])
def test_large_workload_every_slice_against_oracle(precision):
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    (U0, U1), change1 = _golden()
    w = ri.LARGE_N512
    u0 = to_dev(w.initial_state())
    got = {}
    with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=precision) as s:
        for kmax in (0, 1):
            b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, kmax)
            b.arp_set_initial(s.ctx, u0)
            k, ch = b.arp_parareal_solve(s.ctx)
            assert k == kmax
            U = torch.empty((w.slices + 1, 3, w.n_grid // 2 + 1), dtype=torch.complex128, device="cuda")
            b.arp_get_slices(s.ctx, U)
            got[kmax] = (to_host(U), ch)
        info = b.arp_pipeline_info(s.ctx)
    tol = TOL[precision]
    for kmax, ref in ((0, U0), (1, U1)):
        U, _ = got[kmax]
        np.testing.assert_array_equal(U[0], ref[0])
        err = per_state_rel_l2(U[1:], ref[1:])
        assert err.max() <= tol, (kmax, int(err.argmax()) + 1, float(err.max()), info)
    # the convergence quantity of the first iteration (a norm of differences, so
    # compared at the bar of its inputs' error)
    assert abs(got[1][1] / change1 - 1.0) <= 1e-3
