"""The asymptotic coarse solver on a coarser spatial grid (ARP_OPT_COARSE_GRID):
parareal iterates against the FP64 oracle with G = the slow solver on N_c
points (relative L2 <= 1e-10 FP64, <= 1e-5 FP32), and the option's rules."""
import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, to_dev, to_host
from oracle import rsw as o

pytestmark = pytest.mark.gpu


def _iterates(b, p, u0, S, iters, precision, nc, **opts):
    torch = cuda_or_skip()
    its = []
    with b.Solver(p.n_grid, p.eps, p.nu, S, p.dT, p.dt, p.m_quad, precision=precision) as s:
        b.arp_set_option(s.ctx, b.ARP_OPT_COARSE_GRID, nc)
        for key, val in opts.items():
            b.arp_set_option(s.ctx, getattr(b, key), val)
        b.arp_set_initial(s.ctx, to_dev(u0))
        U = torch.empty((S + 1, 3, p.H), dtype=torch.complex128, device="cuda")
        for _ in range(iters + 1):
            b.arp_parareal_iterate(s.ctx)
            b.arp_get_slices(s.ctx, U)
            its.append(to_host(U))
    return its


@pytest.mark.parametrize("nc", [64, 32])
def test_coarse_grid_parareal_matches_oracle(nc):
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(128, 0.02, 1e-4, 0.05, 0.0025, 32)
    u0 = ri.random_spectrum(128, 16, 64.0, 13) * 32.0
    S, iters = 10, 3
    ref = o.parareal(u0, p, S, iters, G=lambda x: o.coarse_step_on_grid(x, p, nc))
    for prec, tol in ((b.ARP_FP64, 1e-10), (b.ARP_FP32, 1e-5)):
        its = _iterates(b, p, u0, S, iters, prec, nc)
        for k in range(iters + 1):
            assert per_state_rel_l2(its[k][1:], ref.iterates[k][1:]).max() <= tol, (prec, k)
        # the modes above the coarse band come from F - G alone: zero after the predictor
        assert np.all(its[0][1:, :, o.kept_modes(nc) + 1:] == 0)


def test_coarse_grid_option_rules():
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(64, 0.02, 1e-4, 0.05, 0.005, 16)
    u0 = ri.random_spectrum(64, 8, 16.0, 3) * 16.0
    with b.Solver(64, p.eps, p.nu, 4, p.dT, p.dt, p.m_quad) as s:
        for bad in (48, 128, 4, 0.5):
            with pytest.raises(b.ArpError) as ei:
                b.arp_set_option(s.ctx, b.ARP_OPT_COARSE_GRID, bad)
            assert ei.value.status == b.ARP_EINVAL
        # the Strang coarse step and the non-cluster chains do not take a coarse grid
        b.arp_set_initial(s.ctx, to_dev(u0))
        for key, val in ((b.ARP_OPT_COARSE_SCHEME, 1), (b.ARP_OPT_CHAIN, 1)):
            b.arp_set_option(s.ctx, b.ARP_OPT_COARSE_GRID, 32)
            b.arp_set_option(s.ctx, key, val)
            with pytest.raises(b.ArpError) as ei:
                b.arp_parareal_iterate(s.ctx)
            assert ei.value.status == b.ARP_EINVAL
            b.arp_set_option(s.ctx, key, 0)
        # batches refuse it
        batch = b.arp_batch_create([s.ctx])
        try:
            b.arp_set_initial(s.ctx, to_dev(u0))
            with pytest.raises(b.ArpError) as ei:
                b.arp_batch_iterate(batch, 1)
            assert ei.value.status == b.ARP_EINVAL
        finally:
            b.arp_batch_destroy(batch)
    # N_c = N is the fine grid itself: the same bits as no option
    same = _iterates(b, p, u0, 4, 2, b.ARP_FP64, 64)
    plain = _iterates(b, p, u0, 4, 2, b.ARP_FP64, 0)
    for a, c in zip(same, plain):
        np.testing.assert_array_equal(a, c)
