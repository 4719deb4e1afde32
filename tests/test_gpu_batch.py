"""Batches of independent problems (arp_batch_*): each problem's iterates equal
those of the same problem run alone, bit for bit, and match the oracle; problems
of different grid sizes, precisions, slice and node counts share one batch, and
problems may join at any level."""
import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip, per_state_rel_l2, to_dev, to_host
from oracle import rsw as o

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5

# (N, eps, nu, slices, dT, dt, M, precision, seed)
PROBLEMS = [
    (64, 1e-2, 1e-4, 8, 0.0625, 1e-3, 32, 0, 1),
    (32, 2e-2, 1e-3, 6, 0.05, 0.0125, 16, 0, 2),
    (64, 5e-3, 1e-4, 4, 0.05, 5e-4, 8, 1, 3),
    (128, 1e-2, 1e-4, 5, 0.04, 2e-3, 32, 1, 4),
    (16, 2e-2, 1e-3, 3, 0.05, 0.0125, 8, 0, 5),
]


def _state(n, seed):
    return ri.random_spectrum(n, min(8, o.kept_modes(n)), 16.0, seed) * 4.0


def _run_alone(b, prob, levels):
    torch = cuda_or_skip()
    n, eps, nu, S, dT, dt, M, prec, seed = prob
    out = []
    with b.Solver(n, eps, nu, S, dT, dt, M, precision=prec) as s:
        b.arp_set_initial(s.ctx, to_dev(_state(n, seed)))
        U = torch.empty((S + 1, 3, n // 2 + 1), dtype=torch.complex128, device="cuda")
        for _ in range(levels):
            b.arp_parareal_iterate(s.ctx)
            b.arp_get_slices(s.ctx, U)
            out.append(to_host(U))
    return out


def _run_batched(b, probs, levels, join_late=()):
    """All problems in one batch; problems listed in join_late get their initial
    state only after the first batched call (they start one level behind)."""
    torch = cuda_or_skip()
    solvers = [b.Solver(*p[:7], precision=p[7]) for p in probs]
    outs = [[] for _ in probs]
    try:
        for i, (s, p) in enumerate(zip(solvers, probs)):
            if i not in join_late:
                b.arp_set_initial(s.ctx, to_dev(_state(p[0], p[8])))
        batch = b.arp_batch_create([s.ctx for s in solvers])
        try:
            for call in range(levels + (1 if join_late else 0)):
                if call == 1:
                    for i in join_late:
                        b.arp_set_initial(solvers[i].ctx, to_dev(_state(probs[i][0], probs[i][8])))
                lv, ch = b.arp_batch_iterate(batch, len(probs))
                for i, (s, p) in enumerate(zip(solvers, probs)):
                    if (i in join_late and call == 0) or len(outs[i]) >= levels:
                        continue
                    U = torch.empty((p[3] + 1, 3, p[0] // 2 + 1), dtype=torch.complex128, device="cuda")
                    b.arp_get_slices(s.ctx, U)
                    outs[i].append(to_host(U))
        finally:
            b.arp_batch_destroy(batch)
    finally:
        for s in solvers:
            s.close()
    return outs


def test_batched_iterates_equal_single_problem_runs_bit_for_bit():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    levels = 3
    batched = _run_batched(b, PROBLEMS, levels)
    for prob, got in zip(PROBLEMS, batched):
        alone = _run_alone(b, prob, levels)
        assert len(got) == levels
        for k in range(levels):
            np.testing.assert_array_equal(got[k], alone[k])


def test_batched_iterates_match_the_oracle():
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    levels = 3
    probs = PROBLEMS[:2] + PROBLEMS[4:] + PROBLEMS[2:4]
    batched = _run_batched(b, probs, levels)
    for prob, got in zip(probs, batched):
        n, eps, nu, S, dT, dt, M, prec, seed = prob
        p = o.Params(n, eps, nu, dT, dt, M)
        ref = o.parareal(_state(n, seed), p, S, levels - 1)
        tol = TOL64 if prec == 0 else TOL32
        for k in range(levels):
            assert per_state_rel_l2(got[k][1:], ref.iterates[k][1:]).max() <= tol, (prob, k)


def test_problem_joining_a_running_batch_and_chain_fallback():
    # problem 1 starts one call late (its predictor runs beside the others'
    # iterations); problem 0 is forced onto its own chain launch (cooperative grid).
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    probs = PROBLEMS[:3]
    levels = 2
    torch = cuda_or_skip()
    solvers = [b.Solver(*p[:7], precision=p[7]) for p in probs]
    try:
        b.arp_set_option(solvers[0].ctx, b.ARP_OPT_CHAIN, 1)
        for i, (s, p) in enumerate(zip(solvers, probs)):
            if i != 1:
                b.arp_set_initial(s.ctx, to_dev(_state(p[0], p[8])))
        batch = b.arp_batch_create([s.ctx for s in solvers])
        lv, ch = b.arp_batch_iterate(batch, 3)
        assert lv == [0, -1, 0] and np.isinf(ch[0]) and np.isnan(ch[1])
        b.arp_set_initial(solvers[1].ctx, to_dev(_state(probs[1][0], probs[1][8])))
        lv, ch = b.arp_batch_iterate(batch, 3)
        assert lv == [1, 0, 1]
        lv, ch = b.arp_batch_iterate(batch, 3)
        assert lv == [2, 1, 2]
        U = torch.empty((probs[1][3] + 1, 3, probs[1][0] // 2 + 1), dtype=torch.complex128, device="cuda")
        b.arp_get_slices(solvers[1].ctx, U)
        late = to_host(U)
        b.arp_batch_destroy(batch)
    finally:
        for s in solvers:
            s.close()
    alone = _run_alone(b, probs[1], 2)
    np.testing.assert_array_equal(late, alone[1])



@pytest.mark.parametrize("n,opts", [(256, [1, 2, 0, 3]), (512, [4, 3, 0, 1])])
def test_batched_members_keep_their_fine_block_size(n, opts):
    # Members of one (N, precision) group that ask for different FP32 fine-sweep
    # schedules (ARP_OPT_FINE_BLOCK) each get the iterates of a solo run with
    # the same option, bit for bit (N = 256: schedules 1-3; N = 512: the
    # radix-16 schedule 4 too).
    torch = cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    base = (n, 1e-2, 1e-4, 4, 0.04, 4e-3, 16, 1, 6)
    probs = [base[:8] + (40 + i,) for i in range(len(opts))]
    alone = []
    for p, v in zip(probs, opts):
        with b.Solver(*p[:7], precision=p[7]) as s:
            b.arp_set_option(s.ctx, b.ARP_OPT_FINE_BLOCK, v)
            b.arp_set_initial(s.ctx, to_dev(_state(p[0], p[8])))
            U = torch.empty((p[3] + 1, 3, p[0] // 2 + 1), dtype=torch.complex128, device="cuda")
            runs = []
            for _ in range(2):
                b.arp_parareal_iterate(s.ctx)
                b.arp_get_slices(s.ctx, U)
                runs.append(to_host(U))
            alone.append(runs)
    solvers = [b.Solver(*p[:7], precision=p[7]) for p in probs]
    try:
        for s, p, v in zip(solvers, probs, opts):
            b.arp_set_option(s.ctx, b.ARP_OPT_FINE_BLOCK, v)
            b.arp_set_initial(s.ctx, to_dev(_state(p[0], p[8])))
        batch = b.arp_batch_create([s.ctx for s in solvers])
        try:
            for k in range(2):
                b.arp_batch_iterate(batch, len(probs))
                for i, (s, p) in enumerate(zip(solvers, probs)):
                    U = torch.empty((p[3] + 1, 3, p[0] // 2 + 1), dtype=torch.complex128, device="cuda")
                    b.arp_get_slices(s.ctx, U)
                    np.testing.assert_array_equal(to_host(U), alone[i][k])
        finally:
            b.arp_batch_destroy(batch)
    finally:
        for s in solvers:
            s.close()
