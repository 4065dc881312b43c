"""Host logic of running the path as independent replicas, one per GPU.

Frames (and their bzip2 blocks) are independent, so N GPUs shard the frames:
rank r compresses its own frames (generator seeds offset by r) and no data
crosses ranks. Throughput of the job = bytes of all ranks / the slowest
rank's time. Only the timing reduction uses a collective.
"""
from __future__ import annotations

import os


def rank_env():
    """(world, rank, local_rank) from the launcher's environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return world, rank, local


def frame_seed(rank: int, i: int, k: int, n_kinds: int) -> int:
    """Seed of frame (repetition i, kind k) on a rank: distinct across ranks,
    rank 0 keeps the single-GPU seeds 1 + k + n_kinds * i."""
    return 1 + k + n_kinds * i + 100003 * rank


def aggregate(local_ms: float, local_bytes: int, device=None):
    """(max over ranks of local_ms, sum over ranks of local_bytes): the job's
    time and bytes. Without an initialised process group, the local values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms), int(local_bytes)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    b = torch.tensor([int(local_bytes)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), int(b.item())


def throughput_mbps(job_ms: float, job_bytes: int) -> float:
    return job_bytes / 1e6 / (job_ms / 1e3) if job_ms > 0 else 0.0
