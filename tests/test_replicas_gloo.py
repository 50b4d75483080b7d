"""The replica aggregation of bench.py on two gloo ranks (CPU): every rank
meshes its own points, the reported throughput counts all ranks' points over
the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local = [2.0, 3.0][rank]
    v, t = bench.replica_value(1_000_000, 10, local, dist)
    q.put((rank, v, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_value_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, v, t in out:
        assert t == pytest.approx(3.0)
        assert v == pytest.approx(2 * 1_000_000 * 10 / 3.0 / 1e6)


def test_replica_value_single():
    import bench

    v, t = bench.replica_value(500, 4, 2.0)
    assert (v, t) == (pytest.approx(500 * 4 / 2.0 / 1e6), 2.0)
