"""The replica path of bench.py under two ranks on the CPU (gloo): the job time is
the slowest rank's, the whole-job throughput counts every replica, and the
reference arm runs on rank 0 alone."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [120.0, 150.0][rank]
        worst = bench.max_over_ranks(ms, world)
        value = bench.job_throughput(1000.0, 10, world, worst)

        class Args:
            gpus, steps, warmup = world, 1, 0
        ref = bench.run_reference(Args(), rank) if rank != 0 else "skipped"
        dist.barrier()
        q.put((rank, worst, value, ref))
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_aggregation_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, worst, value, ref in got:
        assert worst == 150.0                         # the slowest rank's time, on every rank
        assert value == pytest.approx(1000.0 * 10 * 2 / 0.150)
    assert got[1][3] is None                           # rank 1 does no reference work
