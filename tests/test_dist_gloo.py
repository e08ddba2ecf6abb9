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


def _leaver(rank, world, port, out):
    """Rank 1 leaves between two timed steps (after the first reduction, with
    nothing in flight); rank 0's next timing reduction must end with an error
    within the short process-group timeout instead of waiting forever."""
    import datetime

    import torch.distributed as dist

    from paper_2609_36100_gb300.dist import max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    first = max_over_ranks(1.0 + rank)
    if rank == 1:
        out.put((rank, first, "left"))
        out.close()
        out.join_thread()  # the message is written before the process ends
        os._exit(0)  # leaves without destroying the group: the peer sees a dead rank
    try:
        max_over_ranks(3.0)
        out.put((rank, first, "no error"))
    except Exception as e:  # the collective fails: the survivor learns of the loss
        out.put((rank, first, "error: " + type(e).__name__))


def test_rank_leaving_between_steps_is_detected():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaver, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (f, s)) for r, f, s in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
    assert res[1] == (2.0, "left")
    assert res[0][0] == 2.0
    assert res[0][1].startswith("error")
