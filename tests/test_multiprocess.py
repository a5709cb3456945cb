"""Host logic of the multi-GPU bench path on CPU: independent replicas over a
world-size-2 gloo group.  The only collective is the timing reduction (max over
ranks); the data path has none."""

import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # each replica times its own slices; rank 1 is slower
    my_ms = 100.0 + 50.0 * rank
    slowest = bench.reduce_max(my_ms)
    value = bench.replica_throughput(world, 20, slowest)
    dist.barrier()
    q.put((rank, slowest, value))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replicas_take_slowest_rank_gloo():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, slowest, value in res:
        assert slowest == 150.0
        assert abs(value - 2 * 20 / 0.150) < 1e-9


def test_single_process_reduce_is_identity():
    import bench

    assert bench.reduce_max(3.5) == 3.5
    assert bench.replica_throughput(1, 10, 50.0) == 200.0
