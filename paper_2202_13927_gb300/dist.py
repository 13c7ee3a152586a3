"""Sharding of a trial over ranks and the one exchange step (final merge).

Patients are independent and every random draw is keyed by the global
patient id, so rank r simulates a contiguous block of global ids with no
communication.  The only exchange is at the end: the per-patient indicator
records of all ranks are gathered on rank 0 in global-id order and reduced
once (exact integer histograms need the whole population).  Works with any
torch.distributed backend (gloo on CPU tensors, NCCL on CUDA tensors).
"""
from __future__ import annotations

import os


def env_rank_world() -> tuple[int, int, int]:
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_range(rank: int, world: int, n_per_rank: int, base: int = 0) -> tuple[int, int]:
    """Weak scaling: rank r owns global ids [base + r n, base + (r + 1) n)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    first = base + rank * n_per_rank
    return first, first + n_per_rank


def split_range(rank: int, world: int, n_total: int) -> tuple[int, int]:
    """Strong scaling: the n_total ids split into near-equal contiguous blocks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    lo = n_total * rank // world
    hi = n_total * (rank + 1) // world
    return lo, hi


def gather_records(local, rank: int, world: int, group=None):
    """Gather the ranks' uint8 record buffers on rank 0, concatenated in rank
    order (= global-id order for contiguous shards).  The shards may differ in
    size (split_range gives blocks one patient apart): the sizes are exchanged
    first, every buffer is padded to the largest for the gather, and rank 0
    trims each part back to its own size.  Returns the concatenation on rank 0
    and None elsewhere."""
    import torch
    import torch.distributed as dist

    if world == 1:
        return local
    size = torch.tensor([local.numel()], dtype=torch.int64, device=local.device)
    sizes = [torch.zeros_like(size) for _ in range(world)]
    dist.all_gather(sizes, size, group=group)
    sizes = [int(s.item()) for s in sizes]
    longest = max(sizes)
    send = local if local.numel() == longest else torch.cat(
        [local, local.new_zeros(longest - local.numel())])
    parts = [torch.empty_like(send) for _ in range(world)] if rank == 0 else None
    dist.gather(send, parts, dst=0, group=group)
    if rank != 0:
        return None
    return torch.cat([p[:n] for p, n in zip(parts, sizes)])
