"""Parity at the benchmark configurations' own sizes, on samples the oracle can
afford: the N = 1024 precision-sweep workload (1954 steps, M = 128), instances of
the uneven batch generator run as one batch, and a node count too large for the
cluster chain's shared memory (the chain falls back to the cooperative grid)."""
import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, to_dev, to_host
from oracle import rsw as o

pytestmark = pytest.mark.gpu


def _call(fn, s, x):
    torch = cuda_or_skip()
    xin = to_dev(x)
    out = torch.empty_like(xin)
    fn(s.ctx, xin, out)
    return to_host(out)


def test_sweep_workload_sampled():
    # Two states of the N = 1024 workload (1954 steps, M = 128) through contexts
    # of 2 slices and of the workload's 512 slices: the schedule tables pick the
    # FP32 fine sweep by the context's slices per SM, so the 512-slice context
    # runs the schedule the benchmark's sweeps run.
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.SWEEP_N1024
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    x = ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, 2, 77) * 64.0
    fine, avg = o.fine_propagate(x, p), o.nbar(x, p)
    for prec, tol, slices in ((b.ARP_FP64, 1e-10, 2), (b.ARP_FP32, 1e-5, 2), (b.ARP_FP32, 1e-5, w.slices)):
        with b.Solver(w.n_grid, w.eps, w.nu, slices, w.dT, w.dt, w.m_quad, precision=prec) as s:
            assert per_state_rel_l2(_call(b.arp_fine_batch, s, x), fine).max() <= tol, (prec, slices)
            assert per_state_rel_l2(_call(b.arp_coarse_avg, s, x), avg).max() <= tol, (prec, slices)


def test_headline_solve_finite_termination():
    # The benchmark's own call on the N = 1024 workload (512 slices, FP32 bulk,
    # arp_parareal_solve with K_max 5, pipelined where the device allows):
    # after k iterations parareal reproduces the serial fine solution exactly
    # on slices n <= k (Sec. 3), a property that holds at any size, so slices
    # 1..5 must equal F^n(u0) of the oracle within the FP32 bar.
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.SWEEP_N1024
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    u0 = w.initial_state()
    with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=b.ARP_FP32) as s:
        b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, 5)
        b.arp_set_initial(s.ctx, to_dev(u0))
        k, _ = b.arp_parareal_solve(s.ctx)
        U = torch.empty((w.slices + 1, 3, w.n_grid // 2 + 1), dtype=torch.complex128, device="cuda")
        b.arp_get_slices(s.ctx, U)
        got = to_host(U)
    assert k == 5
    assert np.all(np.isfinite(got))
    ref = o.project(u0, w.n_grid)[None]
    for n in range(1, 6):
        ref = o.fine_propagate(ref, p)
        assert per_state_rel_l2(got[n:n + 1], ref).max() <= 1e-5, n


def test_uneven_instances_batched():
    # the generator's first instances whose oracle runs stay short, batched together
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    picks = [w for w in ri.uneven_instances(64) if w.n_grid <= 256 and w.eps >= 2e-3][:3]
    assert len(picks) == 3
    levels = 2
    solvers = [b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=b.ARP_FP32) for w in picks]
    try:
        for s, w in zip(solvers, picks):
            b.arp_set_initial(s.ctx, to_dev(w.initial_state()))
        batch = b.arp_batch_create([s.ctx for s in solvers])
        got = [[] for _ in picks]
        try:
            for _ in range(levels + 1):
                b.arp_batch_iterate(batch, len(picks))
                for i, (s, w) in enumerate(zip(solvers, picks)):
                    U = torch.empty((w.slices + 1, 3, w.n_grid // 2 + 1), dtype=torch.complex128, device="cuda")
                    b.arp_get_slices(s.ctx, U)
                    got[i].append(to_host(U))
        finally:
            b.arp_batch_destroy(batch)
    finally:
        for s in solvers:
            s.close()
    for w, its in zip(picks, got):
        p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
        ref = o.parareal(w.initial_state(), p, w.slices, levels)
        for k in range(levels + 1):
            assert per_state_rel_l2(its[k][1:], ref.iterates[k][1:]).max() <= 1e-5, (w.name, k)


@pytest.mark.parametrize("m", [1024, 4096])
def test_many_quadrature_nodes(m):
    # M = 1024 still fits the cluster chain (64 nodes per CTA); M = 4096 does not and
    # the chain runs as the cooperative grid kernel; both against the oracle
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    n, S = 64, 3
    p = o.Params(n, 0.01, 1e-4, 0.05, 0.005, m)
    u0 = ri.random_spectrum(n, 8, 16.0, 9) * 16.0
    ref = o.parareal(u0, p, S, 1)
    with b.Solver(n, p.eps, p.nu, S, p.dT, p.dt, m) as s:
        b.arp_set_initial(s.ctx, to_dev(u0))
        U = torch.empty((S + 1, 3, n // 2 + 1), dtype=torch.complex128, device="cuda")
        for k in range(2):
            b.arp_parareal_iterate(s.ctx)
            b.arp_get_slices(s.ctx, U)
            assert per_state_rel_l2(to_host(U)[1:], ref.iterates[k][1:]).max() <= 1e-10, k
