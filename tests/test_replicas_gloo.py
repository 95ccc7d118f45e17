"""Replica sharding and the max-over-ranks timing with two gloo CPU ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2107_06381_gb300.replicas import max_over_ranks, shard, sum_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    items = list(range(11))
    mine = shard(items, rank, world)
    total = sum_over_ranks(len(mine))
    slowest = max_over_ranks(1.5 + rank)        # rank 1 is slower
    covered = sum_over_ranks(sum(mine))
    q.put((rank, mine, total, slowest, covered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_cover_everything_once_and_time_is_the_max():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [r[1] for r in res]
    assert sorted(shards[0] + shards[1]) == list(range(11))
    assert not set(shards[0]) & set(shards[1])
    for _, _, total, slowest, covered in res:
        assert total == 11
        assert slowest == 2.5
        assert covered == sum(range(11))


def test_shard_rejects_bad_rank():
    from paper_2107_06381_gb300.replicas import shard
    with pytest.raises(ValueError):
        shard([1, 2], 2, 2)
