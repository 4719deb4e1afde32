"""Slice sharding over ranks (paper_1303_6615_gb300.shard) on the CPU with gloo:
two and three ranks, each owning a contiguous block of slices, with the FP64
oracle's F and G as the propagators.  The sharded iterates (gathered on rank 0)
and changes must be those of the single-process oracle iteration (Eq. 3.1), and
finite termination must hold across block boundaries."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_block_bounds():
    import sys
    sys.path.insert(0, ROOT)
    from paper_1303_6615_gb300.shard import block_bounds
    assert block_bounds(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert block_bounds(4, 4) == [(0, 1), (1, 2), (2, 3), (3, 4)]
    assert block_bounds(5, 1) == [(0, 5)]
    for s in range(1, 30):
        for w in range(1, 6):
            b = block_bounds(s, w)
            assert b[0][0] == 0 and b[-1][1] == s
            assert all(b[i][1] == b[i + 1][0] for i in range(w - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        block_bounds(0, 2)


def _problem():
    import rsw_inputs as ri
    from oracle import rsw as o
    p = o.Params(16, 0.02, 1e-3, 0.05, 0.0125, 8)
    u0 = 2.0 * ri.random_spectrum(16, 5, 16.0, 21)
    return p, u0


def _rank(rank: int, world: int, port: int, slices: int, kmax: int, q) -> None:
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import rsw as o
    from paper_1303_6615_gb300.shard import ShardedParareal
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        p, u0 = _problem()
        F = lambda x: torch.from_numpy(o.fine_propagate(x.numpy(), p))
        G = lambda x: torch.from_numpy(o.coarse_step(x.numpy(), p))
        sp = ShardedParareal(F, G, torch.from_numpy(o.project(u0, p.n_grid)), slices)
        its, changes = [], []
        for _ in range(kmax + 1):
            _, ch = sp.iterate()
            changes.append(ch)
            U = sp.gather()
            its.append(None if U is None else U.numpy())
        q.put((rank, its, changes))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,slices", [(2, 5), (3, 7)])
def test_sharded_iterates_equal_single_process_oracle(world, slices):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import rsw as o
    kmax = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, slices, kmax, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = {}
    for _ in range(world):
        rank, its, changes = q.get(timeout=300)
        got[rank] = (its, changes)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, u0 = _problem()
    ref = o.parareal(u0, p, slices, kmax)
    its, changes = got[0]
    for k in range(kmax + 1):
        d = np.linalg.norm(its[k] - ref.iterates[k]) / np.linalg.norm(ref.iterates[k])
        assert d <= 1e-13, (k, d)
    np.testing.assert_allclose(changes[1:], ref.changes, rtol=1e-9)
    for r in range(1, world):
        assert got[r][0][0] is None                   # only rank 0 gathers
        assert got[r][1][1:] == changes[1:]           # every rank sees the same change
    # finite termination across the block boundaries: U_n^k = F^n(u0) for n <= k
    ser = o.serial_fine(u0, p, slices)
    for k in range(kmax + 1):
        for n in range(min(k, slices) + 1):
            assert np.linalg.norm(its[k][n] - ser[n]) <= 1e-12 * np.linalg.norm(ser[n]), (k, n)
