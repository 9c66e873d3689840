"""Replicas across GPUs: one process per GPU, each running independent chains
with its own Philox key.  The method exchanges two things between replicas:

* at Initialize (Alg. 1), the estimate of p_lambda: every rank must splat
  with the same k0 = p_lambda / (m dt) (Eq. killing-rate-constant), so the
  ranks agree on the mean of p over the union of their initial samples;
* before Resolve (Alg. 3), the FP64 image accumulators and the tour counts:

    image = k0 / (sum over ranks of tourCount) * (sum over ranks of accum)

  which equals Resolve over the union of all ranks' chains."""
from __future__ import annotations

MASK64 = (1 << 64) - 1
GOLDEN64 = 0x9E3779B97F4A7C15


def replica_seed(seed, rank):
    """Philox key of rank `rank`: seed xor rank * 2^64 / phi (distinct for
    every rank, and rank 0 keeps the seed)."""
    return (int(seed) ^ ((int(rank) * GOLDEN64) & MASK64)) & MASK64


def _all_reduce_sum(t, group):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, group=group)
    return t


def agree_p_lambda(p_lambda, n_chains, group=None, device=None):
    """Chain-weighted mean of the ranks' p_lambda estimates, i.e. the mean of p
    over all ranks' initial samples.  ``device`` holds the exchanged tensor
    (a CUDA device under NCCL; None means the CPU, for gloo)."""
    import torch
    t = torch.tensor([float(p_lambda) * int(n_chains), float(n_chains)], dtype=torch.float64, device=device)
    _all_reduce_sum(t, group)
    total = float(t[1].item())
    return float(t[0].item()) / total if total > 0 else 0.0


def init_chains_agreed(r, n_chains, seed, params, group=None, device=None, frame=0):
    """Alg. 1 on every rank with one k0 for all ranks.  ``r`` is a renderer
    (``init_chains(n, seed, params, frame)``, ``counters()`` with
    ``p_lambda``).  When ``params.k0`` > 0 it is used as given; otherwise
    each rank first estimates p_lambda from its own initial samples, the
    ranks agree on the mean, and every rank initialises again with
    k0 = p_lambda / (m dt) given explicitly (the same seed draws the same
    samples, so only the clock sees the new k0).  Returns k0."""
    if params.k0 > 0:
        r.init_chains(n_chains, seed, params, frame)
        return float(params.k0)
    r.init_chains(n_chains, seed, params, frame)
    p_lambda = agree_p_lambda(r.counters()["p_lambda"], n_chains, group, device)
    agreed = type(params).from_buffer_copy(params)
    agreed.k0 = p_lambda / (float(params.m) * float(params.dt))
    r.init_chains(n_chains, seed, agreed, frame)
    return float(agreed.k0)


def merge_and_resolve(accum, tour_count, k0, group=None):
    """accum: FP64 torch tensor (any device the process group supports),
    summed in place over ranks; returns (image, total tour count).  A zero
    total gives a zero image (as Resolve does).  k0 is the one all ranks
    used (see init_chains_agreed)."""
    import torch

    tc = torch.tensor([float(tour_count)], dtype=torch.float64, device=accum.device)
    _all_reduce_sum(accum, group)
    _all_reduce_sum(tc, group)
    total = int(tc.item())
    if total == 0:
        return torch.zeros_like(accum), 0
    return accum * (float(k0) / total), total
