"""The paper's experiments (Sec. 6.2) at reduced size on the GPU: the initial
condition of Eq. 6.4 with the eps = 1 and eps = 1e-1 settings (dT, dt, window,
nodes as printed; grid N = 64 and 10 slices here).  The asymptotic method and
standard parareal with the Strang coarse step match the FP64 oracle iterate by
iterate, and their error against the serial fine solution falls with k, as the
paper's figures report."""
import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, to_dev, to_host
from oracle import rsw as o

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _run(b, e, dT, slices, coarse, window, iters):
    torch = cuda_or_skip()
    n = 64
    its = []
    with b.Solver(n, e.eps, e.nu, slices, dT, e.dt, e.m_quad, T0=window) as s:
        b.arp_set_option(s.ctx, b.ARP_OPT_COARSE_SCHEME, coarse)
        b.arp_set_initial(s.ctx, to_dev(ri.paper_initial_state(n)))
        U = torch.empty((slices + 1, 3, n // 2 + 1), dtype=torch.complex128, device="cuda")
        for _ in range(iters + 1):
            b.arp_parareal_iterate(s.ctx)
            b.arp_get_slices(s.ctx, U)
            its.append(to_host(U))
    return its


def _linf_rel(U, ref, n):
    d = o.physical_linf(U - ref, n)
    return float(np.max(d / o.physical_linf(ref, n)))


@pytest.mark.parametrize("name", ["paper-eps1", "paper-eps1e-1"])
def test_paper_experiment_reduced(name):
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    e = {x.name: x for x in ri.PAPER_EXPERIMENTS}[name]
    n, S, iters = 64, 10, 3
    u0 = ri.paper_initial_state(n)
    for label, dT, coarse, window in (("asymptotic", e.dT, 0, e.window), ("standard", e.standard_dT[0], 1, None)):
        p = o.Params(n, e.eps, e.nu, dT, e.dt, e.m_quad, T0=window)
        G = (lambda x: o.coarse_step_strang(x, p)) if coarse else None
        ref = o.parareal(u0, p, S, iters, G=G)
        its = _run(b, e, dT, S, coarse, window, iters)
        for k in range(iters + 1):
            assert per_state_rel_l2(its[k][1:], ref.iterates[k][1:]).max() <= TOL64, (label, k)
        ser = o.serial_fine(u0, p, S)
        errs = [_linf_rel(U[1:], ser[1:], n) for U in its]
        assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), (label, errs)
