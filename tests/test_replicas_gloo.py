"""Multi-process host logic of the replica launcher, on CPU with gloo
(world size 2): shards cover the work exactly once and the timing reduction
takes the maximum over ranks."""

import os
import socket

import pytest

from paper_2408_16551_gb300 import replicas


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
    try:
        replicas.barrier()
        t = replicas.max_over_ranks(1.5 + rank)          # per-rank "time"
        shards = [replicas.shard_range(1001, r, world) for r in range(world)]
        mine = replicas.shard_range(1001, rank, world)
        halo = replicas.shard_stream_spectra(241, 16, 4096, rank, world)
        q.put((rank, t, shards, mine, halo))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [2.5, 2.5]              # max over ranks, seen by both
    shards = res[0][2]
    covered = [u for (b, e) in shards for u in range(b, e)]
    assert covered == list(range(1001))
    assert res[0][3] == shards[0] and res[1][3] == shards[1]
    (a0, a1, x0, x1), (b0, b1, y0, y1) = res[0][4], res[1][4]
    assert a0 == 0 and a1 == b0 and b1 == 241
    assert x1 == (a1 - 1 + 16) * 4096 and y0 == b0 * 4096    # halo of T-1 frames before rank 1's first spectrum


def test_shard_range_edge_cases():
    assert replicas.shard_range(0, 0, 3) == (0, 0)
    assert replicas.shard_range(2, 2, 3) == (2, 2)
    with pytest.raises(ValueError):
        replicas.shard_range(5, 3, 3)
    assert replicas.max_over_ranks(3.0) == 3.0            # no process group: identity
