"""Host logic of the multi-GPU replica form, on CPU with two gloo ranks: every request is
rendered by exactly one rank, and the job time is the slowest rank's."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2405_13364_gb300 import replicas
    items = list(range(37))
    mine = replicas.shard(items, rank, world)
    t = replicas.max_over_ranks(1.0 + rank, dist)
    n = replicas.sum_over_ranks(len(mine), dist)
    got = [None] * world
    dist.all_gather_object(got, mine)
    dist.barrier()
    if rank == 0:
        q.put((t, n, got))
    dist.destroy_process_group()


def test_replica_sharding_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, n, got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 2.0
    assert n == 37
    flat = sorted(x for part in got for x in part)
    assert flat == list(range(37))
    assert not set(got[0]) & set(got[1])


def test_shard_single_rank():
    from paper_2405_13364_gb300 import replicas
    assert replicas.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert replicas.max_over_ranks(3.5) == 3.5
    assert torch.tensor(1).item() == 1
