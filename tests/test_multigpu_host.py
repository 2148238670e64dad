"""Host logic of the multi-GPU path with world size 2 on the gloo backend
(no GPU): balanced sharding, MAX / SUM over ranks and the aggregate rate."""
import os
import socket

import pytest

from paper_2508_13304_b300.multigpu import aggregate_rate, max_over_ranks, shard, sum_over_ranks


def test_shard_is_balanced_and_complete():
    for n in (0, 1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            parts = [shard(n, r, world) for r in range(world)]
            covered = [i for p in parts for i in p]
            assert covered == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


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
    local_ms = 100.0 + 50.0 * rank                # rank 1 is the slower one
    mine = shard(64, rank, world)
    m = max_over_ranks(local_ms, dist)
    total_units = sum_over_ranks(len(mine), dist)
    dist.barrier()
    q.put((rank, m, total_units, aggregate_rate(total_units, 10, m * 10)))
    dist.destroy_process_group()


def test_two_ranks_on_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, total, rate in res:
        assert m == 150.0
        assert total == 64
        assert abs(rate - 64 / 0.150) < 1e-6
