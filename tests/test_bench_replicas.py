"""Multi-rank path of bench.py on the CPU: independent replicas over gloo (world size 2),
whole-job throughput = all units / slowest rank's time. No GPU is involved."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [100.0, 250.0][rank]
    value, ms = bench.replica_throughput(local_ms, 1.0e6, world)
    out.put((rank, value, ms))
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, value, ms in res:
        assert ms == 250.0  # slowest rank
        assert value == pytest.approx(2 * 1.0e6 / 0.25)


def test_replica_throughput_single_rank():
    import bench

    value, ms = bench.replica_throughput(50.0, 1.0e6, 1)
    assert ms == 50.0 and value == pytest.approx(2.0e7)
