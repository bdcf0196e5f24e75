"""Host-side helpers for running the channeliser as independent replicas,
one process per GPU.

The PFB shards with no exchange: streams (and spectrum ranges of one stream,
given T-1 frames of halo) are independent, so each rank channelises its own
share and nothing crosses ranks on the data path.  Two launchers: whole
streams of a batch dealt to ranks by work (`execute_sharded_batch`), and one
long stream cut into contiguous spectrum ranges (`execute_sharded_stream`).  The only cross-rank step is
timing: a barrier before and after the timed region and the maximum of the
per-rank times.
"""

from __future__ import annotations

import math


def shard_range(n_units: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of n_units for `rank` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad shard arguments")
    base, rem = divmod(n_units, world)
    begin = rank * base + min(rank, rem)
    return begin, begin + base + (1 if rank < rem else 0)


def shard_stream_spectra(S: int, T: int, P: int, rank: int, world: int, hop: int | None = None,
                         granule: int = 1) -> tuple[int, int, int, int]:
    """Split one stream's S spectra across ranks.

    Returns (s_begin, s_end, sample_begin, sample_end): the rank computes
    spectra [s_begin, s_end) from input samples [sample_begin, sample_end).
    Spectrum s reads the P*T samples from s*hop on (hop = P: frames s .. s+T-1),
    so the range holds the share's own frames plus the T-1 frames of halo its
    first spectrum needs.  Shares start on multiples of `granule` spectra (the
    caller picks it so that every slice start keeps the buffer alignment).
    """
    hop = P if hop is None else hop
    if S < 0 or T < 1 or P < 1 or hop < 1 or granule < 1:
        raise ValueError("bad stream shard arguments")
    g0, g1 = shard_range(-(-S // granule), rank, world)
    s0, s1 = min(S, g0 * granule), min(S, g1 * granule)
    if s1 <= s0:
        return s0, s0, s0 * hop, s0 * hop
    return s0, s1, s0 * hop, (s1 - 1) * hop + P * T


def shard_streams(work, rank: int, world: int) -> list[int]:
    """Whole streams of a batch dealt to ranks: largest first, each to the rank
    with the least work so far (ties to the lower rank).  Returns the indices
    `rank` owns, in batch order.  Every rank computes the same deal from the
    same list, so the ranks exchange nothing to agree on it."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad shard arguments")
    work = [int(w) for w in work]
    if any(w < 0 for w in work):
        raise ValueError("negative work")
    load = [0] * world
    owner = [0] * len(work)
    for i in sorted(range(len(work)), key=lambda i: (-work[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += work[i]
    return [i for i in range(len(work)) if owner[i] == rank]


def execute_sharded_batch(entries, rank: int, world: int, stream=None) -> list[int]:
    """Run this rank's share of a batch of (Plan, input, output) entries as one
    pfb_execute_batch call (the work of a stream is its sample count).  Returns
    the indices of the entries run here; the others belong to other ranks."""
    from . import _in_samples, pfb_execute_batch
    mine = shard_streams([_in_samples(x, plan.in_dtype) for plan, x, _ in entries], rank, world)
    if mine:
        pfb_execute_batch([entries[i] for i in mine], stream=stream)
    return mine


def execute_sharded_stream(plan, x, out, rank: int, world: int, stream=None) -> tuple[int, int]:
    """Spectra [s0, s1) of one long stream on this rank: its contiguous share,
    computed from the slice of `x` that starts at the share's first window
    (halo included).  `out` holds the whole stream's spectra [S, P]; only rows
    s0 .. s1-1 are written.  Returns (s0, s1)."""
    from . import PFB_IN_CI8, PFB_IN_R32, _in_samples
    esize = 4 if plan.in_dtype == PFB_IN_R32 else (2 if plan.in_dtype == PFB_IN_CI8 else 8)
    n = _in_samples(x, plan.in_dtype)
    S = plan.out_spectra(n)
    if out.shape[0] < S or out.shape[1] != plan.P:
        raise ValueError("out must hold [S, P] spectra")
    granule = 16 // math.gcd(16, plan.hop * esize)   # slice starts stay 16-byte aligned
    s0, s1, a, b = shard_stream_spectra(S, plan.T, plan.P, rank, world, hop=plan.hop, granule=granule)
    if s1 > s0:
        k = 2 if plan.in_dtype == PFB_IN_CI8 else 1   # int8 input holds (re, im) pairs
        plan.execute(x[k * a:k * b], out=out[s0:s1], stream=stream)
    return s0, s1


def max_over_ranks(value: float, group=None) -> float:
    """Maximum of a per-rank float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def barrier(group=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier(group=group)
