"""arp_parareal_solve pipelined across iterations (ARP_OPT_PIPELINE): the
levels overlap on two SM partitions, and the slices, level and change must be
the level-by-level solve's bit for bit -- for several chunkings (ragged last
chunks, one-link chunks), tolerance stops, solves continued from an earlier
level, the predictor alone, FP32 and FP64 -- and the iterates must match the
FP64 oracle within the FP32 bar.  Configurations outside the pipeline's scope
must fall back to the level-by-level solve."""
import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, to_dev, to_host
from oracle import rsw as o

pytestmark = pytest.mark.gpu


def _solve(b, p, u0, S, precision, pipeline, kmax, tol=0.0, opts=(), continue_to=None):
    """(slices, level, change, pipeline info) after one solve (and a second
    one continued to `continue_to` if given)."""
    torch = cuda_or_skip()
    with b.Solver(p.n_grid, p.eps, p.nu, S, p.dT, p.dt, p.m_quad, precision=precision) as s:
        b.arp_set_option(s.ctx, b.ARP_OPT_PIPELINE, pipeline)
        b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, kmax)
        b.arp_set_option(s.ctx, b.ARP_OPT_TOL, tol)
        for key, val in opts:
            b.arp_set_option(s.ctx, key, val)
        b.arp_set_initial(s.ctx, to_dev(u0))
        k, ch = b.arp_parareal_solve(s.ctx)
        info = b.arp_pipeline_info(s.ctx)
        if continue_to is not None:
            b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, continue_to)
            k, ch = b.arp_parareal_solve(s.ctx)
            info = b.arp_pipeline_info(s.ctx)
        U = torch.empty((S + 1, 3, p.H), dtype=torch.complex128, device="cuda")
        b.arp_get_slices(s.ctx, U)
        # one more level by the level-by-level iteration: the G cache and the
        # previous iterate left by the solve must be the right ones
        k2, ch2 = b.arp_parareal_iterate(s.ctx)
        U2 = torch.empty_like(U)
        b.arp_get_slices(s.ctx, U2)
        assert b.arp_info(s.ctx)["level"] == k2 == k + 1
    return to_host(U), k, ch, info, to_host(U2), ch2


def _params(n=128, S=24, m=32):
    p = o.Params(n, 0.02, 1e-4, 0.05, 0.0025, m)
    u0 = ri.random_spectrum(n, 16, 64.0, 5) * float(n) / 4
    return p, u0, S


def _same(a, c):
    Ua, ka, cha, _, U2a, ch2a = a
    Uc, kc, chc, _, U2c, ch2c = c
    np.testing.assert_array_equal(Ua, Uc)
    np.testing.assert_array_equal(U2a, U2c)
    assert ka == kc and cha == chc and ch2a == ch2c


@pytest.mark.parametrize("chunk", [1, 2, 4, 5, 7, 24, 100])
def test_pipelined_solve_is_the_level_by_level_solve(chunk):
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p, u0, S = _params()
    ref = _solve(b, p, u0, S, b.ARP_FP32, 0, 4)
    assert ref[3]["pipelined"] == 0
    got = _solve(b, p, u0, S, b.ARP_FP32, chunk if chunk >= 2 else 1, 4)
    info = got[3]
    assert info["pipelined"] == 1, info
    assert info["chain_sms"] >= info["cluster"] >= 8 and info["fine_sms"] > 0
    assert info["chunk"] == (min(chunk, S) if chunk >= 2 else min(16, max(4, (S + 15) // 16)))
    _same(got, ref)


@pytest.mark.parametrize("sched", [3, 4])
def test_pipelined_solve_is_the_level_by_level_solve_n512_schedules(sched):
    # the shared-state FP32 schedules (lane pairs; radix-16 plan) at N = 512 on a
    # ragged chunking: pipelined = level by level, bit for bit
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p, u0, S = _params(n=512, S=13, m=16)
    opts = ((b.ARP_OPT_FINE_BLOCK, sched),)
    ref = _solve(b, p, u0, S, b.ARP_FP32, 0, 3, opts=opts)
    got = _solve(b, p, u0, S, b.ARP_FP32, 5, 3, opts=opts)
    assert got[3]["pipelined"] == 1, got[3]
    _same(got, ref)


def test_pipelined_solve_against_the_oracle():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p, u0, S = _params(n=64, S=12, m=16)
    ref = o.parareal(u0, p, S, 3)
    got = _solve(b, p, u0, S, b.ARP_FP32, 3, 3)
    assert got[3]["pipelined"] == 1 and got[1] == 3
    assert per_state_rel_l2(got[0][1:], ref.iterates[3][1:]).max() <= 1e-5


def test_tolerance_stop_and_continued_solves():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p, u0, S = _params(S=20)
    # the changes of the level-by-level iteration
    ref = _solve(b, p, u0, S, b.ARP_FP32, 0, 3)
    changes = []
    torch = cuda_or_skip()
    with b.Solver(p.n_grid, p.eps, p.nu, S, p.dT, p.dt, p.m_quad, precision=b.ARP_FP32) as s:
        b.arp_set_initial(s.ctx, to_dev(u0))
        for _ in range(4):
            changes.append(b.arp_parareal_iterate(s.ctx)[1])
    tol = 0.5 * (changes[1] + changes[2])
    a = _solve(b, p, u0, S, b.ARP_FP32, 4, 10, tol=tol)
    c = _solve(b, p, u0, S, b.ARP_FP32, 0, 10, tol=tol)
    assert a[1] == 2 and a[2] == changes[2] and a[3]["pipelined"] == 1
    _same(a, c)
    # continued: K_max 1, then 3 from there; the predictor alone
    _same(_solve(b, p, u0, S, b.ARP_FP32, 4, 1, continue_to=3), ref)
    _same(_solve(b, p, u0, S, b.ARP_FP32, 4, 0), _solve(b, p, u0, S, b.ARP_FP32, 0, 0))


def test_fp64_cluster_chain_pipelined():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p, u0, S = _params(n=64, S=16, m=16)
    opts = ((b.ARP_OPT_CHAIN, 3),)
    got = _solve(b, p, u0, S, b.ARP_FP64, 4, 3, opts=opts)
    assert got[3]["pipelined"] == 1
    _same(got, _solve(b, p, u0, S, b.ARP_FP64, 0, 3, opts=opts))
    ref = o.parareal(u0, p, S, 3)
    assert per_state_rel_l2(got[0][1:], ref.iterates[3][1:]).max() <= 1e-10


@pytest.mark.parametrize("precision,opts,m", [
    (1, (("ARP_OPT_CHAIN", 1),), 16),
    (1, (("ARP_OPT_COARSE_SCHEME", 1),), 16),
    (1, (("ARP_OPT_COARSE_GRID", 32),), 16),
    (0, (), 32),
], ids=["cooperative-chain", "strang-coarse", "coarse-grid", "fp64-auto-chain-32-nodes"])
def test_out_of_scope_configurations_run_level_by_level(precision, opts, m):
    # (FP64 in automatic mode takes the cooperative grid above 16 nodes)
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p, u0, S = _params(n=64, S=8, m=m)
    o2 = tuple((getattr(b, k), v) for k, v in opts)
    got = _solve(b, p, u0, S, precision, 1, 2, opts=o2)
    assert got[3]["pipelined"] == 0
    _same(got, _solve(b, p, u0, S, precision, 0, 2, opts=o2))


def test_pipeline_option_rules():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p, u0, S = _params(n=64, S=8, m=16)
    with b.Solver(p.n_grid, p.eps, p.nu, S, p.dT, p.dt, p.m_quad, precision=b.ARP_FP32) as s:
        for bad in (-1, 2.5):
            with pytest.raises(b.ArpError) as ei:
                b.arp_set_option(s.ctx, b.ARP_OPT_PIPELINE, bad)
            assert ei.value.status == b.ARP_EINVAL
        with pytest.raises(b.ArpError):
            b.arp_parareal_solve(s.ctx)  # no initial state


@pytest.mark.parametrize("n,S,chunk", [(8, 1, 1), (8, 2, 1), (16, 3, 2), (32, 5, 4), (64, 9, 4)])
def test_pipeline_smallest_problems(n, S, chunk):
    # the smallest grids (no outer FFT stage at N = 8), one to nine slices,
    # chunks of one or more links with a ragged last chunk
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p = o.Params(n, 0.05, 1e-3, 0.1, 0.02, 4)
    u0 = ri.random_spectrum(n, o.kept_modes(n), 4.0, 3) * n
    kmax = min(3, S + 1)
    got = _solve(b, p, u0, S, b.ARP_FP32, chunk if chunk >= 2 else 1, kmax)
    assert got[3]["pipelined"] == 1
    _same(got, _solve(b, p, u0, S, b.ARP_FP32, 0, kmax))
    ref = o.parareal(u0, p, S, kmax)
    assert per_state_rel_l2(got[0][1:], ref.iterates[kmax][1:]).max() <= 1e-5


@pytest.mark.parametrize("scheme", [1, 2], ids=["strang", "ifrk4"])
def test_pipelined_solve_with_other_fine_schemes(scheme):
    # the chunked fine launches run whichever fine scheme the context uses
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p, u0, S = _params(n=64, S=12, m=16)
    opts = ((b.ARP_OPT_FINE_SCHEME, scheme),)
    got = _solve(b, p, u0, S, b.ARP_FP32, 4, 3, opts=opts)
    assert got[3]["pipelined"] == 1
    _same(got, _solve(b, p, u0, S, b.ARP_FP32, 0, 3, opts=opts))


def test_fp64_automatic_chain_with_few_nodes_is_pipelined():
    # FP64 with at most 16 nodes chains in the cluster, so its solve is pipelined
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    p, u0, S = _params(n=64, S=12, m=10)
    got = _solve(b, p, u0, S, b.ARP_FP64, 4, 3)
    assert got[3]["pipelined"] == 1
    _same(got, _solve(b, p, u0, S, b.ARP_FP64, 0, 3))
    ref = o.parareal(u0, p, S, 3)
    assert per_state_rel_l2(got[0][1:], ref.iterates[3][1:]).max() <= 1e-10


def test_concurrent_solves_on_two_threads():
    # two host threads solve on their own contexts at once; the shared SM
    # partition is pushed under its lock, and each thread's slices are the
    # ones a sequential solve gives
    import threading
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    cases = [_params(n=64, S=12, m=16), _params(n=128, S=16, m=16)]
    seq = [_solve(b, p, u0, S, b.ARP_FP32, 1, 3)[0] for p, u0, S in cases]
    out, errors = [None, None], []

    def run(i):
        try:
            p, u0, S = cases[i]
            dev = torch.device("cuda", 0)
            torch.cuda.set_device(dev)
            for _ in range(3):
                with b.Solver(p.n_grid, p.eps, p.nu, S, p.dT, p.dt, p.m_quad, precision=b.ARP_FP32) as s:
                    b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, 3)
                    b.arp_set_initial(s.ctx, to_dev(u0))
                    b.arp_parareal_solve(s.ctx)
                    U = torch.empty((S + 1, 3, p.H), dtype=torch.complex128, device="cuda")
                    b.arp_get_slices(s.ctx, U)
                    out[i] = to_host(U)
        except Exception as exc:  # reported below
            errors.append(exc)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=120)
    assert not any(t.is_alive() for t in threads), "a solving thread did not finish"
    assert not errors, errors
    for i in range(2):
        np.testing.assert_array_equal(out[i], seq[i])
