"""GPU parity of the Strang-splitting paths (Algorithm 3; standard parareal with
the Strang coarse step, Sec. 6.2) and of the integrating-factor RK4 fine solver
(Sec. 6.2's comparator) through the C ABI against the FP64 oracle: relative
L2 <= 1e-10 (FP64) and <= 1e-5 (FP32 bulk), per state."""
import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, to_dev, to_host
from oracle import rsw as o

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


def _solver(b, p, slices, precision=0, fine=0, coarse=0):
    s = b.Solver(p.n_grid, p.eps, p.nu, slices, p.dT, p.dt, p.m_quad, precision=precision)
    b.arp_set_option(s.ctx, b.ARP_OPT_FINE_SCHEME, fine)
    b.arp_set_option(s.ctx, b.ARP_OPT_COARSE_SCHEME, coarse)
    return s


def _call(fn, s, x):
    torch = cuda_or_skip()
    xin = to_dev(x)
    out = torch.empty_like(xin)
    fn(s.ctx, xin, out)
    return to_host(out)


def _states(n, count, seed, amp):
    return amp * ri.random_batch(n, min(8, o.kept_modes(n)), 16.0, count, seed)


@pytest.mark.parametrize("n,batch", [(8, 3), (16, 4), (64, 5), (128, 3), (256, 2), (512, 2), (1024, 2), (2048, 1)])
def test_strang_fine_sweep_fp64_and_fp32(n, batch):
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    # FP64 on a strongly nonlinear state (physical amplitude ~12); FP32 on one of
    # amplitude ~3.  The first is ill-conditioned for single precision itself: the
    # oracle's Strang solver with the nonlinearity evaluated in float32 already
    # departs from its float64 result by 1e-4 at N = 512 (4e-5 at N = 2048), while
    # at amplitude ~3 that departure is 2e-8.
    p = o.Params(n, 0.02, 1e-3 if n <= 256 else 1e-6, 0.02, 0.004, 8)
    for prec, tol, amp in ((b.ARP_FP64, TOL64, 2.0), (b.ARP_FP32, TOL32, 0.5)):
        x = _states(n, batch, 500 + n, float(n) * amp)
        ref = o.strang_propagate(x, p)
        with _solver(b, p, batch, prec, fine=1) as s:
            got = _call(b.arp_fine_batch, s, x)
        assert per_state_rel_l2(got, ref).max() <= tol, prec


def test_strang_fine_sweep_large_workload_sample():
    # the large workload's sizes (N = 512, 391 steps of dt = 1e-4 per slice), 3 slices
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.LARGE_N512
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    x = ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, 3, 21) * 16.0
    ref = o.strang_propagate(x, p)
    for prec, tol in ((b.ARP_FP64, TOL64), (b.ARP_FP32, TOL32)):
        with _solver(b, p, 3, prec, fine=1) as s:
            assert per_state_rel_l2(_call(b.arp_fine_batch, s, x), ref).max() <= tol, prec


def test_strang_coarse_step_and_options():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(64, 0.01, 1e-4, 0.0625, 1e-3, 32)
    x = _states(64, 6, 31, 8.0)
    ref = o.coarse_step_strang(x, p)
    for prec, tol in ((b.ARP_FP64, TOL64), (b.ARP_FP32, TOL32)):
        with _solver(b, p, 6, prec, coarse=1) as s:
            assert per_state_rel_l2(_call(b.arp_coarse_step, s, x), ref).max() <= tol, prec
            # the time average itself does not depend on the coarse scheme
            avg = _call(b.arp_coarse_avg, s, x)
            assert per_state_rel_l2(avg, o.nbar(x, p)).max() <= tol
            for key, bad in ((b.ARP_OPT_FINE_SCHEME, 3), (b.ARP_OPT_COARSE_SCHEME, 2)):
                with pytest.raises(b.ArpError) as ei:
                    b.arp_set_option(s.ctx, key, bad)
                assert ei.value.status == b.ARP_EINVAL
            # batches take the default schemes only
            b.arp_set_initial(s.ctx, to_dev(x[0]))
            batch = b.arp_batch_create([s.ctx])
            try:
                with pytest.raises(b.ArpError) as ei:
                    b.arp_batch_iterate(batch, 1)
                assert ei.value.status == b.ARP_EINVAL
            finally:
                b.arp_batch_destroy(batch)


def test_strang_geostrophic_state_only_decays():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    from test_oracle_coarse import _geostrophic_state
    p = o.Params(32, 0.01, 1e-3, 0.0625, 1e-3, 16)
    u0 = _geostrophic_state(32, 4)[None]
    decay = np.exp(-p.nu * np.arange(p.H) ** 4 * p.dT)
    with _solver(b, p, 1, fine=1, coarse=1) as s:
        np.testing.assert_allclose(_call(b.arp_fine_batch, s, u0)[0], decay * u0[0], atol=1e-13)
        np.testing.assert_allclose(_call(b.arp_coarse_step, s, u0)[0], decay * u0[0], atol=1e-13)


def _gpu_parareal(b, p, u0, slices, iters, precision, fine, coarse):
    torch = cuda_or_skip()
    its = []
    with _solver(b, p, slices, precision, fine, coarse) as s:
        b.arp_set_initial(s.ctx, to_dev(u0))
        U = torch.empty((slices + 1, 3, p.H), dtype=torch.complex128, device="cuda")
        for _ in range(iters + 1):
            b.arp_parareal_iterate(s.ctx)
            b.arp_get_slices(s.ctx, U)
            its.append(to_host(U))
    return its


@pytest.mark.parametrize("fine", [0, 1], ids=["etdrk4", "strang"])
def test_standard_parareal_matches_oracle(fine):
    # standard parareal (Strang coarse step of the full equation), fine = ETDRK4 or Strang
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(64, 0.05, 1e-4, 0.1, 0.005, 16)
    u0 = ri.random_spectrum(64, 8, 16.0, 77) * 8.0
    S, iters = 12, 3
    F = (lambda x: o.strang_propagate(x, p)) if fine else None
    ref = o.parareal(u0, p, S, iters, F=F, G=lambda x: o.coarse_step_strang(x, p))
    for prec, tol in ((b.ARP_FP64, TOL64), (b.ARP_FP32, TOL32)):
        its = _gpu_parareal(b, p, u0, S, iters, prec, fine, 1)
        for k in range(iters + 1):
            assert per_state_rel_l2(its[k][1:], ref.iterates[k][1:]).max() <= tol, (prec, k)


def test_asymptotic_parareal_with_strang_fine_matches_oracle():
    # Algorithm 4 as printed: the asymptotic coarse solver with the Strang fine solver
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.SMALL_N64
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    u0 = w.initial_state()
    ref = o.parareal(u0, p, w.slices, 2, F=lambda x: o.strang_propagate(x, p))
    for prec, tol in ((b.ARP_FP64, TOL64), (b.ARP_FP32, TOL32)):
        its = _gpu_parareal(b, p, u0, w.slices, 2, prec, 1, 0)
        for k in range(3):
            assert per_state_rel_l2(its[k][1:], ref.iterates[k][1:]).max() <= tol, (prec, k)


def test_standard_parareal_finite_termination_on_gpu():
    # U_n^k equals the serial fine solution for n <= k (Eq. 3.1), GPU against GPU
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(32, 0.05, 1e-4, 0.1, 0.01, 8)
    u0 = ri.random_spectrum(32, 8, 16.0, 5) * 6.0
    S = 5
    its = _gpu_parareal(b, p, u0, S, S, b.ARP_FP64, 0, 1)
    with _solver(b, p, 1) as s:
        ser = [o.project(u0, 32)]
        for _ in range(S):
            ser.append(_call(b.arp_fine_batch, s, ser[-1][None])[0])
    ser = np.stack(ser)
    scale = np.max(np.abs(ser))
    for k, U in enumerate(its):
        for n in range(min(k, S) + 1):
            assert np.max(np.abs(U[n] - ser[n])) <= 1e-12 * scale, (k, n)


# ----------------------------------------------------------- integrating-factor RK4

@pytest.mark.parametrize("n,batch", [(8, 3), (64, 5), (256, 2), (512, 2), (2048, 1)])
def test_ifrk4_fine_sweep_fp64_and_fp32(n, batch):
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(n, 0.02, 1e-3 if n <= 256 else 1e-6, 0.02, 0.004, 8)
    for prec, tol, amp in ((b.ARP_FP64, TOL64, 2.0), (b.ARP_FP32, TOL32, 0.5)):
        x = _states(n, batch, 700 + n, float(n) * amp)
        ref = o.ifrk4_propagate(x, p)
        with _solver(b, p, batch, prec, fine=2) as s:
            got = _call(b.arp_fine_batch, s, x)
        assert per_state_rel_l2(got, ref).max() <= tol, prec


def test_ifrk4_geostrophic_and_parareal():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    from test_oracle_coarse import _geostrophic_state
    p = o.Params(32, 0.01, 1e-3, 0.0625, 1e-3, 16)
    u0 = _geostrophic_state(32, 4)[None]
    decay = np.exp(-p.nu * np.arange(p.H) ** 4 * p.dT)
    with _solver(b, p, 1, fine=2) as s:
        np.testing.assert_allclose(_call(b.arp_fine_batch, s, u0)[0], decay * u0[0], atol=1e-13)
    # the asymptotic method with the integrating-factor fine solver
    w = ri.SMALL_N64
    q = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    v0 = w.initial_state()
    ref = o.parareal(v0, q, w.slices, 2, F=lambda x: o.ifrk4_propagate(x, q))
    for prec, tol in ((b.ARP_FP64, TOL64), (b.ARP_FP32, TOL32)):
        its = _gpu_parareal(b, q, v0, w.slices, 2, prec, 2, 0)
        for k in range(3):
            assert per_state_rel_l2(its[k][1:], ref.iterates[k][1:]).max() <= tol, (prec, k)
