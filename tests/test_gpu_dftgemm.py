"""The DFT-as-GEMM precisions on the library's own tcgen05 tensor-core kernel.

1. The split-precision GEMM itself (arp_gemm_check) against an FP64 matrix
   product of the same FP32 inputs, on shapes that span several 128 x 128
   tiles with ragged edges in every dimension.
2. ARP_TF32X3 and ARP_BF16X3 (split into two TF32 / three BF16 parts): the
   batched time average, the coarse step, the lock-step ETDRK4 fine sweep and
   the parareal iteration against the FP64 oracle at the FP32 bar, 1e-5
   relative L2.
3. ARP_BF16X2 (two BF16 parts, about 16 significant bits per operand) is
   measured, not held to the bar: its error is reported, and the test only
   checks that the three-part split is the more accurate one."""
import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, to_dev, to_host
from oracle import rsw as o

pytestmark = pytest.mark.gpu

TOL = 1e-5
PARITY = [(2, "tf32x3"), (4, "bf16x3")]


def _solver(b, p, slices, precision):
    return b.Solver(p.n_grid, p.eps, p.nu, slices, p.dT, p.dt, p.m_quad, precision=precision)


def _call(fn, s, x):
    torch = cuda_or_skip()
    xin = to_dev(x)
    out = torch.empty_like(xin)
    fn(s.ctx, xin, out)
    return to_host(out)


@pytest.mark.parametrize("prec,split_err", [(2, 1e-6), (3, 3e-5), (4, 1e-6)], ids=["tf32x3", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("m,n,k", [(128, 128, 32), (300, 200, 100), (512, 1000, 384), (77, 5, 1030)])
def test_split_gemm_against_fp64_product(prec, split_err, m, n, k):
    # relative Frobenius error of C against the exact product of the FP32 inputs:
    # the split's operand error plus the FP32 accumulation of k terms of random
    # sign, which grows like sqrt(k) 2^-24 relative to the result
    bound = split_err + 16.0 * np.sqrt(k) * 2.0 ** -24
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((m, k)).astype(np.float32)
    B = rng.standard_normal((n, k)).astype(np.float32)
    C = torch.full((n, m), float("nan"), dtype=torch.float32, device="cuda")
    b.arp_gemm_check(prec, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C)
    got = to_host(C).astype(np.float64)
    ref = B.astype(np.float64) @ A.astype(np.float64).T
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"gemm prec {prec} {m}x{n}x{k}: {err:.2e}")
    assert np.all(np.isfinite(got)) and err <= bound


def test_split_gemm_identity_and_exact_integers():
    # small integers are exact in every input type: the tiles must be placed
    # exactly (a transposed operand, a shifted k step or a wrong row would show)
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    rng = np.random.default_rng(5)
    m, n, k = 256, 384, 192
    A = rng.integers(-3, 4, size=(m, k)).astype(np.float32)
    B = rng.integers(-3, 4, size=(n, k)).astype(np.float32)
    for prec in (2, 3, 4):
        C = torch.empty((n, m), dtype=torch.float32, device="cuda")
        b.arp_gemm_check(prec, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C)
        np.testing.assert_array_equal(to_host(C), B @ A.T)


@pytest.mark.parametrize("prec,name", PARITY, ids=[p[1] for p in PARITY])
@pytest.mark.parametrize("n,m,batch", [(64, 32, 5), (256, 64, 3), (512, 20, 5), (1024, 8, 2)])
def test_dft_gemm_time_average_and_coarse_step(prec, name, n, m, batch):
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(n, 0.01, 1e-4, 0.05, 1e-3, m)
    x = ri.random_batch(n, min(16, o.kept_modes(n)), 64.0, batch, 40 + n) * float(n)
    with _solver(b, p, batch, prec) as s:
        avg = _call(b.arp_coarse_avg, s, x)
        g = _call(b.arp_coarse_step, s, x)
    e_avg = per_state_rel_l2(avg, o.nbar(x, p)).max()
    e_g = per_state_rel_l2(g, o.coarse_step(x, p)).max()
    print(f"dft {name} N={n} M={m}: avg {e_avg:.2e} step {e_g:.2e}")
    assert e_avg <= TOL and e_g <= TOL


@pytest.mark.parametrize("prec,name", PARITY, ids=[p[1] for p in PARITY])
def test_dft_gemm_fine_sweep_and_parareal(prec, name):
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.SMALL_N64
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    x = ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, w.slices, 3) * 8.0
    with _solver(b, p, w.slices, prec) as s:
        got = _call(b.arp_fine_batch, s, x)
    e_f = per_state_rel_l2(got, o.fine_propagate(x, p)).max()
    u0 = w.initial_state()
    ref = o.parareal(u0, p, w.slices, 2)
    its = []
    with _solver(b, p, w.slices, prec) as s:
        b.arp_set_initial(s.ctx, to_dev(u0))
        U = torch.empty((w.slices + 1, 3, p.H), dtype=torch.complex128, device="cuda")
        for _ in range(3):
            b.arp_parareal_iterate(s.ctx)
            b.arp_get_slices(s.ctx, U)
            its.append(to_host(U))
    e_p = max(per_state_rel_l2(its[k][1:], ref.iterates[k][1:]).max() for k in range(3))
    print(f"dft {name}: fine {e_f:.2e} parareal {e_p:.2e}")
    assert e_f <= TOL and e_p <= TOL


def test_dft_gemm_large_time_average_sample():
    # the large workload's sizes (N = 512, M = 64) on 3 states: 192 column
    # groups, 6 column tiles of the inverse GEMM, 3 row tiles of the forward one
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.LARGE_N512
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    x = ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, 3, 31) * 64.0
    ref = o.nbar(x, p)
    for prec, name in PARITY:
        with _solver(b, p, 3, prec) as s:
            e = per_state_rel_l2(_call(b.arp_coarse_avg, s, x), ref).max()
        print(f"dft {name} large time average: {e:.2e}")
        assert e <= TOL


def test_dft_gemm_large_fine_sample_and_batch_rule():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    w = ri.LARGE_N512
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    x = ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, 2, 21) * 16.0
    ref = o.fine_propagate(x, p)
    with _solver(b, p, 2, b.ARP_TF32X3) as s:
        e = per_state_rel_l2(_call(b.arp_fine_batch, s, x), ref).max()
        print(f"dft tf32x3 large fine: {e:.2e}")
        assert e <= TOL
        b.arp_set_initial(s.ctx, to_dev(x[0]))
        batch = b.arp_batch_create([s.ctx])
        try:
            with pytest.raises(b.ArpError) as ei:
                b.arp_batch_iterate(batch, 1)
            assert ei.value.status == b.ARP_EINVAL
        finally:
            b.arp_batch_destroy(batch)


def test_bf16x2_is_measured_not_held_to_the_bar():
    # two BF16 parts keep about 16 significant bits: the time average lands near
    # 1e-5, around the FP32 bar, so this precision is reported, not claimed
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(512, 0.01, 1e-4, 0.05, 1e-3, 16)
    x = ri.random_batch(512, 16, 64.0, 2, 552) * 512.0
    ref = o.nbar(x, p)
    err = {}
    for prec in (b.ARP_BF16X2, b.ARP_BF16X3):
        with _solver(b, p, 2, prec) as s:
            got = _call(b.arp_coarse_avg, s, x)
        assert np.all(np.isfinite(got))
        err[prec] = per_state_rel_l2(got, ref).max()
    print(f"time average N=512: bf16x2 {err[b.ARP_BF16X2]:.2e}, bf16x3 {err[b.ARP_BF16X3]:.2e}")
    assert err[b.ARP_BF16X3] * 10 <= err[b.ARP_BF16X2]
