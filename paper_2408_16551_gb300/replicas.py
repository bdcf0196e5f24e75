"""Host-side helpers for running the channeliser as independent replicas,
one process per GPU.

The PFB shards with no exchange: streams (and spectrum ranges of one stream,
given T-1 frames of halo) are independent, so each rank channelises its own
share and nothing crosses ranks on the data path.  The only cross-rank step is
timing: a barrier before and after the timed region and the maximum of the
per-rank times.
"""

from __future__ import annotations


def shard_range(n_units: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of n_units for `rank` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad shard arguments")
    base, rem = divmod(n_units, world)
    begin = rank * base + min(rank, rem)
    return begin, begin + base + (1 if rank < rem else 0)


def shard_stream_spectra(S: int, T: int, P: int, rank: int, world: int) -> tuple[int, int, int, int]:
    """Split one stream's S spectra across ranks.

    Returns (s_begin, s_end, sample_begin, sample_end): the rank computes
    spectra [s_begin, s_end) from input samples [sample_begin, sample_end),
    which includes the T-1 frames of halo its first spectrum needs.
    """
    s0, s1 = shard_range(S, rank, world)
    if s1 <= s0:
        return s0, s1, s0 * P, s0 * P
    return s0, s1, s0 * P, (s1 - 1 + T) * P


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
