"""Ensemble members sharded over ranks, one GPU per rank.

Members are independent runs, so every rank steps and diagnoses its own
contiguous block of members with no communication; once per diagnostic event
the per-member statistics (``Lattice.subvolume_balance_batch``: FP64
[members, sizes, 15, 2]) are gathered in global member order.  This is host
plumbing over ``torch.distributed`` (any backend: tensors go to the current
CUDA device for NCCL and stay on the host otherwise); every step of the
simulation and of the diagnostic runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np


def shard(n_members: int, world_size: int, rank: int) -> range:
    """The contiguous block of global member indices owned by ``rank``: the
    first ``n_members % world_size`` ranks take one member more."""
    if n_members < 0 or world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("need n_members >= 0, world_size >= 1 and 0 <= rank < world_size")
    base, extra = divmod(n_members, world_size)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def gather_member_stats(stats, group=None) -> np.ndarray:
    """All ranks' per-member statistics, concatenated in rank order (global
    member order for ``shard``'s blocks), returned on every rank.  Shards may
    have different member counts (including none); every rank must pass the
    same trailing shape.  Without an initialised process group, or with one
    rank, the input is returned unchanged."""
    import torch
    import torch.distributed as dist
    stats = np.ascontiguousarray(stats, dtype=np.float64)
    if not dist.is_available() or not dist.is_initialized():
        return stats
    ws = dist.get_world_size(group)
    if ws == 1:
        return stats
    dev = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend(group) == "nccl" else torch.device("cpu")
    n = torch.tensor([stats.shape[0]], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(n) for _ in range(ws)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    rows = max(counts)
    pad = torch.zeros((rows,) + stats.shape[1:], dtype=torch.float64, device=dev)
    if stats.shape[0]:
        pad[:stats.shape[0]] = torch.from_numpy(stats).to(dev)
    parts = [torch.empty_like(pad) for _ in range(ws)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)]).cpu().numpy()
