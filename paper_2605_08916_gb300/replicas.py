"""Replicas across GPUs: one process per GPU, each running independent chains
with its own Philox key; the only exchange of the method is the merge of the
FP64 image accumulators and the tour counts before Resolve (Alg. 3):

    image = k0 / (sum over ranks of tourCount) * (sum over ranks of accum)

which equals Resolve over the union of all ranks' chains."""
from __future__ import annotations

MASK64 = (1 << 64) - 1
GOLDEN64 = 0x9E3779B97F4A7C15


def replica_seed(seed, rank):
    """Philox key of rank `rank`: seed xor rank * 2^64 / phi (distinct for
    every rank, and rank 0 keeps the seed)."""
    return (int(seed) ^ ((int(rank) * GOLDEN64) & MASK64)) & MASK64


def merge_and_resolve(accum, tour_count, k0, group=None):
    """accum: FP64 torch tensor (any device the process group supports),
    summed in place over ranks; returns (image, total tour count).  A zero
    total gives a zero image (as Resolve does)."""
    import torch
    import torch.distributed as dist

    tc = torch.tensor([float(tour_count)], dtype=torch.float64, device=accum.device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(accum, group=group)
        dist.all_reduce(tc, group=group)
    total = int(tc.item())
    if total == 0:
        return torch.zeros_like(accum), 0
    return accum * (float(k0) / total), total
