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


# ---- stream-sharded launchers: the host logic, with the oracle doing the arithmetic ----

def test_shard_streams_deal():
    """Every stream goes to exactly one rank, the deal is the same on every rank,
    and the loads differ by at most the largest stream."""
    from paper_2408_16551_gb300 import synth
    work = [s.n_samples for s in synth.config_c4(256)]
    for world in (1, 2, 3, 4, 8):
        deals = [replicas.shard_streams(work, r, world) for r in range(world)]
        owned = sorted(i for d in deals for i in d)
        assert owned == list(range(len(work)))
        assert all(d == sorted(d) for d in deals)
        loads = [sum(work[i] for i in d) for d in deals]
        assert max(loads) - min(loads) <= max(work)
        assert deals == [replicas.shard_streams(work, r, world) for r in range(world)]
    assert replicas.shard_streams([], 0, 2) == []
    assert replicas.shard_streams([5], 1, 2) == []          # more ranks than streams: idle rank
    with pytest.raises(ValueError):
        replicas.shard_streams([1, -1], 0, 2)
    with pytest.raises(ValueError):
        replicas.shard_streams([1], 2, 2)


@pytest.mark.parametrize("S,T,P,hop,granule", [(241, 16, 4096, 4096, 1), (1021, 4, 16, 16, 1),
                                               (1000, 8, 64, 32, 1), (37, 3, 4, 4, 2), (0, 4, 16, 16, 1),
                                               (5, 16, 256, 128, 4)])
def test_shard_stream_spectra_cover(S, T, P, hop, granule):
    """Shares tile [0, S) in order, start on granule multiples, and each sample
    range is exactly the span of its spectra's windows."""
    for world in (1, 2, 3, 7):
        nxt = 0
        for r in range(world):
            s0, s1, a, b = replicas.shard_stream_spectra(S, T, P, r, world, hop=hop, granule=granule)
            assert s0 == nxt and s1 >= s0
            assert s0 % granule == 0 or s0 == S
            if s1 > s0:
                assert a == s0 * hop and b == (s1 - 1) * hop + P * T
            else:
                assert a == b
            nxt = s1
        assert nxt == S


@pytest.mark.parametrize("P,T,hop,world", [(16, 4, 16, 3), (8, 5, 8, 2), (32, 3, 8, 4)])
def test_sharded_stream_halo_oracle(P, T, hop, world):
    """The shards' spectra, each computed from its own input slice (halo
    included), equal the whole stream's spectra bit for bit (FP64 oracle,
    same arithmetic per spectrum)."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(P * 100 + T)
    N = P * 61 + 5                                          # ragged tail
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    h = oracle.prototype(P, T)
    whole = oracle.pfb_hop(x, P, T, h, hop)
    S = whole.shape[0]
    parts = []
    for r in range(world):
        s0, s1, a, b = replicas.shard_stream_spectra(S, T, P, r, world, hop=hop)
        if s1 > s0:
            part = oracle.pfb_hop(x[a:b], P, T, h, hop)
            assert part.shape[0] == s1 - s0
            parts.append(part)
    assert np.array_equal(np.concatenate(parts), whole)


def _shard_worker(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P, T = 16, 4
        rng = np.random.default_rng(11)                     # same input on every rank
        N = P * 200
        x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        h = oracle.prototype(P, T)
        S = oracle.num_spectra(N, P, T)
        s0, s1, a, b = replicas.shard_stream_spectra(S, T, P, rank, world)
        mine = oracle.pfb(x[a:b], P, T, h) if s1 > s0 else np.zeros((0, P), complex)
        gathered = [None] * world
        dist.all_gather_object(gathered, (s0, s1, mine))
        if rank == 0:
            gathered.sort(key=lambda g: g[0])
            got = np.concatenate([g[2] for g in gathered])
            q.put((rank, bool(np.array_equal(got, oracle.pfb(x, P, T, h))), [g[:2] for g in gathered]))
        else:
            q.put((rank, None, None))
    finally:
        dist.destroy_process_group()


def test_sharded_stream_two_ranks_gloo():
    """World size 2: each rank channelises its share of one stream from its
    halo'd slice; the shares gathered on rank 0 equal the whole output."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in procs], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res[0][1] is True
    assert res[0][2] == [(0, 99), (99, 197)]


class _StubPlan:
    """Stands in for a Plan in host-logic tests: records execute() calls."""

    def __init__(self, P, T, in_dtype, hop=None):
        self.P, self.T, self.in_dtype, self.hop = P, T, in_dtype, hop or P
        self.calls = []

    def out_spectra(self, n):
        L = self.P * self.T
        return 0 if n < L else (n - L) // self.hop + 1

    def execute(self, x, out=None, stream=None):
        self.calls.append((x, out))


@pytest.mark.parametrize("P,T,in_dtype,hop,world", [(1024, 16, 1, None, 3), (1024, 16, 1, 512, 4),
                                                    (4, 3, 2, None, 3), (16, 4, 0, None, 5)])
def test_execute_sharded_stream_host_logic(P, T, in_dtype, hop, world):
    """Each rank hands the plan the input slice of its spectra's windows (int8
    input counts two values per sample) and the matching output rows; slice
    starts keep 16-byte alignment."""
    import torch
    import paper_2408_16551_gb300 as pkg
    esize = {pkg.PFB_IN_R32: 4, pkg.PFB_IN_C64: 8, pkg.PFB_IN_CI8: 2}[in_dtype]
    k = 2 if in_dtype == pkg.PFB_IN_CI8 else 1
    n = P * (T + 41) + 3
    x = torch.arange(k * n)                                # element index = value
    plan = _StubPlan(P, T, in_dtype, hop)
    S = plan.out_spectra(n)
    out = torch.zeros((S, P))
    rows = []
    for r in range(world):
        s0, s1 = replicas.execute_sharded_stream(plan, x, out, r, world)
        rows.append((s0, s1))
    assert rows[0][0] == 0 and rows[-1][1] == S
    assert all(rows[i][1] == rows[i + 1][0] for i in range(world - 1))
    calls = [c for c in plan.calls]
    assert len(calls) == sum(1 for s0, s1 in rows if s1 > s0)
    for (xs, os_), (s0, s1) in zip(calls, [r for r in rows if r[1] > r[0]]):
        a, b = int(xs[0]) // k, (int(xs[-1]) + 1) // k       # sample range of the slice
        assert a == s0 * plan.hop and b == (s1 - 1) * plan.hop + P * T
        assert (a * esize) % 16 == 0
        assert plan.out_spectra(b - a) == s1 - s0
        assert os_.shape[0] == s1 - s0 and os_.data_ptr() == out[s0].data_ptr()


def test_execute_sharded_batch_host_logic(monkeypatch):
    """Each rank passes exactly its dealt entries to one batch call."""
    import torch
    import paper_2408_16551_gb300 as pkg
    calls = []
    monkeypatch.setattr(pkg, "pfb_execute_batch", lambda entries, stream=None: calls.append(list(entries)))
    sizes = [5000, 70, 1 << 16, 3000, 12, 40000, 999]
    entries = [(_StubPlan(16, 4, pkg.PFB_IN_C64), torch.empty(m, dtype=torch.complex64), None) for m in sizes]
    world = 3
    ran = []
    for r in range(world):
        mine = replicas.execute_sharded_batch(entries, r, world)
        assert mine == replicas.shard_streams(sizes, r, world)
        ran += mine
        assert [id(e) for e in calls[-1]] == [id(entries[i]) for i in mine]
    assert sorted(ran) == list(range(len(sizes)))
    assert len(calls) == world
