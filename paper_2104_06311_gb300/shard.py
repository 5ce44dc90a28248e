"""Channel sharding of the batched form across ranks (one GPU per rank).

WDM channels are independent receivers: a batch splits across ranks with no
exchange on the data path.  Each rank runs its own rx_batch over a subset of
the channels chosen to balance the work (longest-processing-time-first on a
per-channel cost of sample-times times the format's equaliser step weight), and
the per-channel error counts are merged once, after the data path, by a sum over
ranks.  Host logic only: the channels' DSP runs in the library's kernels.
"""
from __future__ import annotations

# an equaliser update step of 16QAM weighs this many QPSK steps (the batched
# equaliser's team-size model uses the same weight)
STEP_WEIGHT_16QAM = 1.075


def channel_cost(n_samples: int, mod_bits: int) -> float:
    """Work of one channel, in QPSK sample-time units."""
    return float(n_samples) * (STEP_WEIGHT_16QAM if mod_bits == 4 else 1.0)


def shard_channels(costs, world: int) -> list[list[int]]:
    """Partition channel indices over `world` ranks, balancing the summed cost.

    Longest processing time first: channels in decreasing cost (ties: lower
    index first) go to the rank with the smallest load so far (ties: lower
    rank).  Deterministic, so every rank computes the same partition without
    communicating.  Each rank's list is in increasing channel order.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda c: (-costs[c], c))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for c in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(c)
        load[r] += costs[c]
    return [sorted(p) for p in parts]


def merge_counts(counts, n_channels: int, rank_channels, dist=None, device="cpu"):
    """Per-channel (errors, bits) of this rank's channels -> every channel's, on every rank.

    counts[i] belongs to channel rank_channels[i]; the result lists all
    n_channels entries (a channel no rank owns stays (0, 0)).  With torch
    distributed initialised, the counts are summed over ranks (all_reduce);
    without it this rank's counts are the result.
    """
    import torch
    t = torch.zeros((n_channels, 2), dtype=torch.int64, device=device)
    for (e, b), ch in zip(counts, rank_channels):
        t[ch, 0] = int(e)
        t[ch, 1] = int(b)
    if dist is not None and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [(int(e), int(b)) for e, b in t.cpu().tolist()]
