"""World-size-2 gloo run (CPU) of the multi-rank bench logic: ensemble
members shard disjointly and completely, and the timing reduction takes the
maximum over ranks."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2609_36100_gb300.dist import max_over_ranks, shard, sum_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard(64, rank, world)
    allv = [None] * world
    dist.all_gather_object(allv, mine)
    t = max_over_ranks(1.0 + rank * 0.5)
    s = sum_over_ranks(len(mine))
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, allv, t, s))


def test_two_rank_sharding_and_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, allv, t, s in res:
        flat = sorted(i for part in allv for i in part)
        assert flat == list(range(64))
        assert not set(allv[0]) & set(allv[1])
        assert t == pytest.approx(1.5)
        assert s == 64


def test_shard_rejects_bad_rank():
    from paper_2609_36100_gb300.dist import shard
    with pytest.raises(ValueError):
        shard(4, 2, 2)
