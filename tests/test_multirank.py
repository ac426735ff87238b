"""The N-replica path of bench.py (replicas only: the density does not shard
across GPUs here, every rank runs the same workload): two `gloo` ranks on the
CPU check the rendezvous, the barrier, the max over ranks and the whole-job
rate, as a two-GPU run would use them."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms = 100.0 + 50.0 * rank          # rank 1 is the slowest
        worst = bench.max_over_ranks(world, ms)
        value = bench.replica_value(world, 1e12, worst)
        bench.barrier(world)
        q.put((rank, worst, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_replica_rate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, worst, value in got:
        assert worst == 150.0                       # both ranks see the slowest time
        assert value == pytest.approx(2 * 1e12 / 0.150 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1, 12.5) == 12.5
    assert bench.replica_value(1, 2e9, 1000.0) == pytest.approx(2.0)
