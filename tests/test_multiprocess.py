"""The multi-rank host path on CPU: two gloo ranks (127.0.0.1) run the
bench's timing aggregation (max over ranks) and the batch sharding (every
genome on exactly one rank, balanced by length)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class _G:
    def __init__(self, n, length):
        self.name = n
        self.length = length


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1807_00205_gb300 import batch
    ms = bench.aggregate_max_ms(10.0 + 5.0 * rank, world)
    items = [_G(k, 1000 + 37 * k * k) for k in range(23)]
    mine = [g.name for g in batch.shard(items, rank, world)]
    dist.barrier()
    q.put((rank, ms, mine))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert all(ms == 15.0 for _, ms, _ in out)  # the slowest rank's time on every rank
    a, b = out[0][2], out[1][2]
    assert sorted(a + b) == list(range(23)) and not set(a) & set(b)
    la = sum(1000 + 37 * k * k for k in a)
    lb = sum(1000 + 37 * k * k for k in b)
    assert abs(la - lb) / (la + lb) < 0.2
