"""The multi-GPU bench path is replicas only (independent simulations per rank, no
data-path collective); its max-time / summed-work aggregation runs here on CPU
with two gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = bench.aggregate(elapsed=1.0 + rank, work=[10.0 * rank, 5.0, 3.0], world=world, device="cpu")
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        elapsed, work = res[r]
        assert elapsed == 2.0                 # the slowest rank
        assert work == [10.0, 10.0, 6.0]      # summed over ranks


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate(3.5, [1, 2], 1) == (3.5, [1.0, 2.0])
