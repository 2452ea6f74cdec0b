"""Multi-rank host logic on CPU (gloo, world size 2): sharding, barrier, max-over-ranks timing."""

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1205_6872_gb300 import replicas


def test_shard_covers_everything_once():
    for n in (0, 1, 5, 256, 257):
        for world in (1, 2, 3, 4, 8):
            seen = []
            sizes = []
            for r in range(world):
                a, b = replicas.shard(n, r, world)
                seen.extend(range(a, b))
                sizes.append(b - a)
            assert seen == list(range(n))
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = replicas.env_ranks()
        replicas.barrier()
        t = replicas.reduce_max(1.5 + rank)      # per-rank "time"
        s = replicas.reduce_sum(10.0 * (rank + 1))
        a, b = replicas.shard(256, r, w)
        q.put((rank, w, r, lr, t, s, a, b))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for rank, w, r, lr, t, s, a, b in got:
        assert (w, r, lr) == (2, rank, rank)
        assert t == 2.5          # max over ranks
        assert s == 30.0
    assert (got[0][6], got[0][7], got[1][6], got[1][7]) == (0, 128, 128, 256)


def test_single_process_identity():
    assert replicas.reduce_max(3.25) == 3.25
    replicas.barrier()
