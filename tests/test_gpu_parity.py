"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Bar: relative L2 <= 1e-10 for the FP64 path and <= 1e-5
for the FP32 path (bulk arithmetic in FP32, tables and phases from FP64,
parareal correction and norm in FP64)."""
import math

import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, rel_l2, to_dev, to_host
from oracle import rsw as o

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


def _solver(p: o.Params, slices: int, precision: int = 0):
    from paper_1303_6615_gb300 import binding as b
    s = b.Solver(p.n_grid, p.eps, p.nu, slices, p.dT, p.dt, p.m_quad, precision=precision,
                 T0=p.T0, F=None if p.F == 1.0 else p.F)
    return s


def _states(n, count, seed, amp=1.0, cutoff=None):
    K = o.kept_modes(n)
    c = min(8, K) if cutoff is None else cutoff
    return amp * ri.random_batch(n, c, 16.0, count, seed)


def _gpu_call(fn, solver, x: np.ndarray) -> np.ndarray:
    torch = cuda_or_skip()
    xin = to_dev(x)
    out = torch.empty_like(xin)
    fn(solver.ctx, xin, out)
    return to_host(out)


# ---------------------------------------------------------------- fine propagator

@pytest.mark.parametrize("n,batch", [(8, 3), (16, 5), (32, 7), (64, 5), (128, 3), (256, 2), (1024, 2), (2048, 1)])
def test_fine_fp64_grid_sizes(n, batch):
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(n, 0.02, 1e-3 if n <= 256 else 1e-6, 0.02, 0.005, 8)
    x = _states(n, batch, 100 + n, amp=float(n) * 2.0)
    with _solver(p, max(batch, 1)) as s:
        got = _gpu_call(b.arp_fine_batch, s, x)
    ref = o.fine_propagate(x, p)
    assert per_state_rel_l2(got, ref).max() <= TOL64


def test_fine_fp64_small_workload():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.SMALL_N64
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    x = ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, w.slices, 0) * 8.0
    with _solver(p, w.slices) as s:
        got = _gpu_call(b.arp_fine_batch, s, x)
    ref = o.fine_propagate(x, p)
    assert per_state_rel_l2(got, ref).max() <= TOL64


def test_fine_fp64_large_instance_sampled():
    # N = 512, eps = 1e-3, dt = 1e-4 (391 steps per slice), 3 sampled states
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.LARGE_N512
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    x = ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, 3, 7) * 16.0
    with _solver(p, w.slices) as s:
        got = _gpu_call(b.arp_fine_batch, s, x)
    ref = o.fine_propagate(x, p)
    assert per_state_rel_l2(got, ref).max() <= TOL64


def test_fine_projection_empty_batch_and_mean_height():
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    n = 64
    p = o.Params(n, 0.01, 1e-4, 0.0625, 1e-3, 32)
    x = _states(n, 4, 5, amp=10.0)
    junk = x.copy()
    rng = np.random.default_rng(0)
    K = o.kept_modes(n)
    junk[:, :, K + 1:] = rng.standard_normal(junk[:, :, K + 1:].shape)
    junk[:, :, 0] += 0.25j
    with _solver(p, 4) as s:
        clean = _gpu_call(b.arp_fine_batch, s, x)
        dirty = _gpu_call(b.arp_fine_batch, s, junk)
        e = torch.empty((0, 3, n // 2 + 1), dtype=torch.complex128, device="cuda")
        b.arp_fine_batch(s.ctx, e, e)
    np.testing.assert_array_equal(clean, dirty)
    assert np.all(clean[:, :, K + 1:] == 0) and np.all(clean[:, :, 0].imag == 0)
    # mean height: the k = 0 coefficient of h is carried through bit for bit
    np.testing.assert_array_equal(clean[:, 2, 0], x[:, 2, 0].real)


def test_fine_geostrophic_state_only_decays():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    n = 64
    p = o.Params(n, 0.01, 1e-4, 0.0625, 1e-3, 32)
    rng = np.random.default_rng(4)
    K = o.kept_modes(n)
    u = np.zeros((1, 3, n // 2 + 1), dtype=complex)
    for k in range(K + 1):
        a = rng.standard_normal() + (1j * rng.standard_normal() if k else 0)
        u[0, :, k] = a * np.array([0, 1j * k, 1]) / math.sqrt(1 + k * k)
    with _solver(p, 1) as s:
        got = _gpu_call(b.arp_fine_batch, s, u)
    decay = np.exp(-p.nu * np.arange(p.H) ** 4 * p.dT)
    np.testing.assert_allclose(got, decay * u, atol=1e-13)


# ---------------------------------------------------------------- time average and slow solver

@pytest.mark.parametrize("n,m,batch,T0", [(8, 4, 3, None), (64, 32, 5, None), (64, 31, 2, 11.0), (512, 64, 2, None)])
def test_coarse_avg_fp64(n, m, batch, T0):
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(n, 0.01 if n < 512 else 1e-3, 1e-4, 0.0625 if n < 512 else 10 / 256, 1e-3, m, T0=T0)
    x = _states(n, batch, 40 + n, amp=float(n))
    with _solver(p, batch) as s:
        got = _gpu_call(b.arp_coarse_avg, s, x)
    ref = o.nbar(x, p)
    assert per_state_rel_l2(got, ref).max() <= TOL64


@pytest.mark.parametrize("n,m,batch", [(16, 8, 3), (64, 32, 5), (512, 64, 2)])
def test_coarse_step_fp64(n, m, batch):
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(n, 0.01 if n < 512 else 1e-3, 1e-4, 0.0625 if n < 512 else 10 / 256, 1e-3, m)
    x = _states(n, batch, 60 + n, amp=float(n))
    with _solver(p, batch) as s:
        got = _gpu_call(b.arp_coarse_step, s, x)
    ref = o.coarse_step(x, p)
    assert per_state_rel_l2(got, ref).max() <= TOL64


def test_coarse_results_do_not_depend_on_batch():
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    n = 64
    p = o.Params(n, 0.01, 1e-4, 0.0625, 1e-3, 32)
    x = _states(n, 6, 9, amp=32.0)
    with _solver(p, 6) as s:
        all6 = _gpu_call(b.arp_coarse_step, s, x)
        one = _gpu_call(b.arp_coarse_step, s, x[3:4])
    np.testing.assert_array_equal(all6[3:4], one)


# ---------------------------------------------------------------- parareal

def _gpu_parareal(p, u0, slices, iters, precision=0, chain=0):
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    its, changes = [], []
    with _solver(p, slices, precision) as s:
        b.arp_set_option(s.ctx, b.ARP_OPT_CHAIN, chain)
        b.arp_set_initial(s.ctx, to_dev(u0))
        U = torch.empty((slices + 1, 3, p.H), dtype=torch.complex128, device="cuda")
        for _ in range(iters + 1):
            k, ch = b.arp_parareal_iterate(s.ctx)
            b.arp_get_slices(s.ctx, U)
            its.append(to_host(U))
            changes.append(ch)
    return its, changes


@pytest.mark.parametrize("chain", [0, 1, 2, 3], ids=["auto", "cooperative", "launches", "cluster"])
def test_parareal_small_workload_fp64(chain):
    w = ri.SMALL_N64
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    u0 = w.initial_state()
    its, changes = _gpu_parareal(p, u0, w.slices, w.k_max, chain=chain)
    ref = o.parareal(u0, p, w.slices, w.k_max)
    assert len(its) == len(ref.iterates)
    for k, (g, r) in enumerate(zip(its, ref.iterates)):
        assert per_state_rel_l2(g[1:], r[1:]).max() <= TOL64, k
        np.testing.assert_array_equal(g[0], o.project(u0, w.n_grid))
    assert math.isinf(changes[0])
    # the change is a norm of differences of nearly equal FP64 iterates: its
    # absolute rounding floor is about 1e-13 (relative to the iterate's norm)
    np.testing.assert_allclose(changes[1:], ref.changes, rtol=1e-6, atol=1e-13)


def test_parareal_finite_termination_gpu():
    n, S = 16, 4
    p = o.Params(n, 0.02, 1e-3, 0.05, 0.0125, 8)
    u0 = 2.0 * ri.random_spectrum(n, 5, 16.0, 21)
    its, _ = _gpu_parareal(p, u0, S, S)
    ser = o.serial_fine(u0, p, S)
    for k, U in enumerate(its):
        for m in range(0, min(k, S) + 1):
            assert rel_l2(U[m], ser[m]) <= TOL64, (k, m)


def test_parareal_requires_initial_state():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(16, 0.02, 1e-3, 0.05, 0.0125, 8)
    with _solver(p, 2) as s:
        with pytest.raises(b.ArpError) as ei:
            b.arp_parareal_iterate(s.ctx)
        assert ei.value.status == b.ARP_EINVAL


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_parareal_large_instance_sampled(precision):
    # N = 512, 256 slices, M = 64, the bench's launch configuration: the first
    # three slices of the predictor and of the first iteration, computed by the
    # oracle one by one from u0.
    w = ri.LARGE_N512
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    u0 = w.initial_state()
    tol = TOL64 if precision == 0 else TOL32
    its, changes = _gpu_parareal(p, u0, w.slices, 1, precision=precision)
    G = lambda x: o.coarse_step(x, p)
    F = lambda x: o.fine_propagate(x, p)
    U0 = [o.project(u0, p.n_grid)]
    for _ in range(3):
        U0.append(G(U0[-1]))
    Fs = F(np.stack(U0[:3]))
    U1 = [U0[0]]
    for n_ in range(3):
        U1.append(G(U1[-1]) + Fs[n_] - G(U0[n_]))
    for n_ in range(1, 4):
        assert rel_l2(its[0][n_], U0[n_]) <= tol, n_
        assert rel_l2(its[1][n_], U1[n_]) <= tol, n_
    assert np.isfinite(changes[1])
    # mean height through the whole chain
    np.testing.assert_allclose(its[1][:, 2, 0].real, u0[2, 0].real, rtol=0, atol=1e-15 if precision == 0 else 1e-9)


# ---------------------------------------------------------------- FP32 bulk path

def test_fine_fp32_small_workload_and_large_sample():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    for w, count, amp in ((ri.SMALL_N64, 16, 8.0), (ri.LARGE_N512, 3, 16.0)):
        p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
        x = ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, count, 11) * amp
        with _solver(p, count, precision=b.ARP_FP32) as s:
            got = _gpu_call(b.arp_fine_batch, s, x)
        ref = o.fine_propagate(x, p)
        assert per_state_rel_l2(got, ref).max() <= TOL32, w.name


@pytest.mark.parametrize("n", [64, 128, 256, 512, 1024, 2048])
def test_fine_fp32_schedules(n):
    # The FP32 fine sweep has four schedules (ARP_OPT_FINE_BLOCK 1 = N/4 threads,
    # 2 = N/2 threads, 3 = N/8 threads with lane pairs and shared stage values for
    # N >= 256, 4 = N/8 threads with radix-16 stages for 512 <= N <= 2048; 0
    # takes the tuned default per grid size; 3 and 4 fall back to the default
    # where they do not apply).  Each is deterministic, each meets the FP32 bar
    # against the oracle, they differ only by FP32 rounding, and the default is
    # one of them.
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(n, 0.02, 1e-4 if n <= 256 else 1e-6, 0.02, 0.002, 8)
    x = _states(n, 5, 300 + n, amp=float(n) * 2.0 if n <= 1024 else 1024.0)
    got, sched = {}, {}
    with _solver(p, 5, precision=b.ARP_FP32) as s:
        with pytest.raises(b.ArpError) as ei:
            b.arp_set_option(s.ctx, b.ARP_OPT_FINE_BLOCK, 5)
        assert ei.value.status == b.ARP_EINVAL
        for v in (0, 1, 2, 3, 4):
            b.arp_set_option(s.ctx, b.ARP_OPT_FINE_BLOCK, v)
            sched[v] = b.arp_info(s.ctx)["fine_schedule"]
            got[v] = _gpu_call(b.arp_fine_batch, s, x)
            np.testing.assert_array_equal(_gpu_call(b.arp_fine_batch, s, x), got[v])
    assert sched[1] == 1 and sched[3] == (3 if n >= 256 else sched[0])
    assert sched[4] == (4 if 512 <= n <= 2048 else sched[0])
    assert any(np.array_equal(got[0], got[v]) for v in (1, 2, 3, 4))
    for v in (2, 3, 4):
        assert per_state_rel_l2(got[1], got[v]).max() <= 1e-6, v
    ref = o.fine_propagate(x, p)
    for v in (1, 2, 3, 4):
        assert per_state_rel_l2(got[v], ref).max() <= TOL32, v


def test_coarse_fp32():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.SMALL_N64
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    x = ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, 4, 3) * 8.0
    with _solver(p, 4, precision=b.ARP_FP32) as s:
        avg = _gpu_call(b.arp_coarse_avg, s, x)
        g = _gpu_call(b.arp_coarse_step, s, x)
    assert per_state_rel_l2(avg, o.nbar(x, p)).max() <= TOL32
    assert per_state_rel_l2(g, o.coarse_step(x, p)).max() <= TOL32


@pytest.mark.parametrize("chain", [0, 1, 3], ids=["auto", "cooperative", "cluster"])
def test_parareal_small_workload_fp32(chain):
    from paper_1303_6615_gb300 import binding as b
    w = ri.SMALL_N64
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    u0 = w.initial_state()
    cuda_or_skip()
    its, _ = _gpu_parareal(p, u0, w.slices, w.k_max, precision=b.ARP_FP32, chain=chain)
    ref = o.parareal(u0, p, w.slices, w.k_max)
    for k, (g, r) in enumerate(zip(its, ref.iterates)):
        assert per_state_rel_l2(g[1:], r[1:]).max() <= TOL32, k


# ---------------------------------------------------------------- failure detection

@pytest.mark.parametrize("hook,precision", [(1, 0), (2, 0), (2, 1)],
                         ids=["cooperative-grid", "cluster-fp64", "cluster-fp32"])
def test_chain_barrier_timeout_is_reported_and_context_stays_usable(hook, precision):
    # Test hook, one chain launch: 1 -- block 0 of the cooperative grid skips its
    # first barrier arrival; 2 -- CTA 0 of the cluster does not send its first
    # partial sums.  Every wait on them gives up after about a second.
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.SMALL_N64
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    u0 = w.initial_state()
    with _solver(p, w.slices, precision) as s:
        b.arp_set_initial(s.ctx, to_dev(u0))
        b.arp_set_option(s.ctx, b.ARP_OPT_TEST_SKIP_ARRIVAL, hook)
        with pytest.raises(b.ArpError) as ei:
            b.arp_parareal_iterate(s.ctx)
        assert ei.value.status == b.ARP_ETIMEOUT
        # the CUDA context is intact: restart the iteration and compare with the oracle
        b.arp_set_initial(s.ctx, to_dev(u0))
        b.arp_parareal_iterate(s.ctx)
        U = torch.empty((w.slices + 1, 3, p.H), dtype=torch.complex128, device="cuda")
        b.arp_get_slices(s.ctx, U)
        got = to_host(U)
    ref = o.parareal(u0, p, w.slices, 0)
    assert per_state_rel_l2(got[1:], ref.iterates[0][1:]).max() <= (TOL64 if precision == 0 else TOL32)
