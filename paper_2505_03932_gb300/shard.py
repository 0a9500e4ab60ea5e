"""Multi-GPU sharding of batched reprojection (one process per GPU).

Frames are independent (every target pixel of every exposure is computed on its own), so a batch
shards by frame with no exchange on the data path: rank r of N takes frames r, r+N, r+2N, ...
and runs dfr_reproject_batch on its share. The only collectives are for timing and bookkeeping:
a barrier, and the maximum step time over ranks (the slowest rank bounds the job).
"""
from __future__ import annotations


def frames_for_rank(n_frames: int, rank: int, world: int):
    """Indices of the frames rank ``rank`` of ``world`` processes (round robin)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(range(rank, n_frames, world))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (value itself if none)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
