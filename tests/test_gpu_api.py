"""The C ABI's iteration and buffer calls on the GPU: arp_parareal_solve against
explicit arp_parareal_iterate calls (K_max and tolerance stopping, bit for bit),
host and device buffers, arp_info, and the smallest problems."""
import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, to_dev, to_host
from oracle import rsw as o

pytestmark = pytest.mark.gpu


def _small():
    w = ri.SMALL_N64
    return w, o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad), w.initial_state()


def _iterate(b, w, u0, levels, precision=0):
    torch = cuda_or_skip()
    out, changes = [], []
    with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=precision) as s:
        b.arp_set_initial(s.ctx, to_dev(u0))
        U = torch.empty((w.slices + 1, 3, w.n_grid // 2 + 1), dtype=torch.complex128, device="cuda")
        for _ in range(levels + 1):
            k, ch = b.arp_parareal_iterate(s.ctx)
            changes.append(ch)
            b.arp_get_slices(s.ctx, U)
            out.append(to_host(U))
    return out, changes


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_solve_equals_explicit_iterations(precision):
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w, p, u0 = _small()
    its, changes = _iterate(b, w, u0, 4, precision)
    H = w.n_grid // 2 + 1
    # K_max = 3, no tolerance: predictor + 3 iterations
    with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=precision) as s:
        b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, 3)
        b.arp_set_initial(s.ctx, to_dev(u0))
        k, ch = b.arp_parareal_solve(s.ctx)
        assert k == 3 and ch == changes[3]
        U = torch.empty((w.slices + 1, 3, H), dtype=torch.complex128)  # host buffer
        b.arp_get_slices(s.ctx, U)
        np.testing.assert_array_equal(U.numpy(), its[3])
        assert b.arp_info(s.ctx)["level"] == 3
        # solving again continues from the current level up to the new K_max
        b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, 4)
        k, ch = b.arp_parareal_solve(s.ctx)
        assert k == 4 and ch == changes[4]
    # a tolerance between two consecutive changes stops at the first level at or below it
    tol = 0.5 * (changes[1] + changes[2])
    with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=precision) as s:
        b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, 10)
        b.arp_set_option(s.ctx, b.ARP_OPT_TOL, tol)
        b.arp_set_initial(s.ctx, to_dev(u0))
        k, ch = b.arp_parareal_solve(s.ctx)
        assert k == 2 and ch == changes[2] and ch <= tol
    # K_max = 0: the predictor only
    with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=precision) as s:
        b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, 0)
        b.arp_set_initial(s.ctx, to_dev(u0))
        assert b.arp_parareal_solve(s.ctx)[0] == 0
        U = torch.empty((w.slices + 1, 3, H), dtype=torch.complex128, device="cuda")
        b.arp_get_slices(s.ctx, U)
        np.testing.assert_array_equal(to_host(U), its[0])


def test_info_and_host_initial_state():
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w, p, u0 = _small()
    with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad) as s:
        info = b.arp_info(s.ctx)
        assert info == {"N": 64, "H": 33, "K": 21, "slices": 16, "M": 32, "steps": 63, "level": -1, "precision": 0,
                        "fine_schedule": 1}
        b.arp_set_initial(s.ctx, torch.from_numpy(u0))  # pageable host memory
        b.arp_parareal_iterate(s.ctx)
        U = torch.empty((w.slices + 1, 3, 33), dtype=torch.complex128)
        b.arp_get_slices(s.ctx, U)
    ref = o.parareal(u0, p, w.slices, 0)
    assert per_state_rel_l2(U.numpy()[1:], ref.iterates[0][1:]).max() <= 1e-10


@pytest.mark.parametrize("n,m,slices", [(8, 2, 1), (8, 3, 2), (16, 2, 3)])
def test_smallest_problems(n, m, slices):
    # the smallest grid, node count and slice count through the whole iteration
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(n, 0.05, 1e-3, 0.1, 0.02, m)
    u0 = ri.random_spectrum(n, o.kept_modes(n), 4.0, 3) * n
    ref = o.parareal(u0, p, slices, 2)
    for prec, tol in ((0, 1e-10), (1, 1e-5)):
        its = []
        torch = cuda_or_skip()
        with b.Solver(n, p.eps, p.nu, slices, p.dT, p.dt, m, precision=prec) as s:
            b.arp_set_initial(s.ctx, to_dev(u0))
            U = torch.empty((slices + 1, 3, n // 2 + 1), dtype=torch.complex128, device="cuda")
            for _ in range(3):
                b.arp_parareal_iterate(s.ctx)
                b.arp_get_slices(s.ctx, U)
                its.append(to_host(U))
        for k in range(3):
            assert per_state_rel_l2(its[k][1:], ref.iterates[k][1:]).max() <= tol, (prec, k)


def test_alu_peak_probe():
    # the measured FMA peak the bench reports beside the nominal one: positive, of
    # the right order for the part (FP32 far above FP64), other precisions refused
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    f32 = b.arp_alu_peak(b.ARP_FP32)
    f64 = b.arp_alu_peak(b.ARP_FP64)
    assert 10.0 < f32 < 200.0 and 0.1 < f64 < 10.0 and f32 > 8 * f64
    with pytest.raises(b.ArpError) as ei:
        b.arp_alu_peak(b.ARP_TF32X3)
    assert ei.value.status == b.ARP_EINVAL
