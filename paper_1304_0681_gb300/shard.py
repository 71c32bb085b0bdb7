"""Sharding a batch over GPUs: one process per GPU, no exchange on the data path.

Stage E aligns every (read, candidate) pair on its own, and the paper runs
whole batches of reads through Stages D and E in parallel (§3.4).  So a batch
splits into contiguous groups of reads, and each group takes all of its
candidate windows along.  The best hit of a read needs every candidate of
that read, so a group never splits a read.  The split balances DP cells
(read length times window length, summed over a group's pairs), which is
what the score and traceback passes cost.

The only collective is at the end of a run: it reduces the counters the
caller reports, summing the units and taking the slowest rank's time.
"""
from __future__ import annotations

import numpy as np


def read_costs(read_lengths, cand_offsets, window_lengths) -> np.ndarray:
    """DP cells of each read: m_r times the summed lengths of its windows."""
    read_lengths = np.asarray(read_lengths, np.int64)
    cand_offsets = np.asarray(cand_offsets, np.int64)
    window_lengths = np.asarray(window_lengths, np.int64)
    wsum = np.zeros(len(window_lengths) + 1, np.int64)
    np.cumsum(window_lengths, out=wsum[1:])
    per_read = wsum[cand_offsets[1:]] - wsum[cand_offsets[:-1]]
    return read_lengths * per_read


def cell_balanced_bounds(read_lengths, cand_offsets, window_lengths, world_size: int) -> np.ndarray:
    """Read boundaries b[0] = 0 <= b[1] <= ... <= b[W] = n_reads.

    Rank k aligns reads b[k] .. b[k+1] and their candidates.  Each b[k]
    (0 < k < W) is the read boundary whose cell prefix is nearest
    k/W of the total.  A rank's share is therefore within one read's cost
    of total/W, and a rank may get no reads at all when there are fewer
    reads than ranks."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    cost = read_costs(read_lengths, cand_offsets, window_lengths)
    n = len(cost)
    prefix = np.zeros(n + 1, np.int64)
    np.cumsum(cost, out=prefix[1:])
    total = int(prefix[-1])
    bounds = np.zeros(world_size + 1, np.int64)
    bounds[-1] = n
    for k in range(1, world_size):
        target = total * k / world_size
        hi = int(np.searchsorted(prefix, target, side="left"))
        hi = min(hi, n)
        lo = max(hi - 1, 0)
        bounds[k] = lo if abs(prefix[lo] - target) <= abs(prefix[hi] - target) else hi
    return np.maximum.accumulate(bounds)


def reduce_run(units: float, seconds: float, group=None) -> tuple:
    """(sum of units over ranks, max of seconds over ranks).

    Without torch.distributed initialised this is the identity.  The tensors
    live on the CPU for gloo and on the current CUDA device for nccl."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(units), float(seconds)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    s = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(s, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()), float(s.item())
