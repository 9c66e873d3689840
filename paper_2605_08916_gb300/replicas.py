"""Replicas across GPUs: one process per GPU, each running independent chains
with its own Philox key.  The method exchanges two things between replicas:

* at Initialize (Alg. 1), the estimate of p_lambda: every rank must splat
  with the same k0 = p_lambda / (m dt) (Eq. killing-rate-constant), so the
  ranks pool their initial samples: the library's sum of p over each rank's
  initial samples and their count are summed over ranks, and the library
  turns the totals into k0;
* before Resolve (Alg. 3), the FP64 image accumulators and the tour counts
  (64-bit integers), summed over ranks; the library then resolves

    image = k0 / (sum over ranks of tourCount) * (sum over ranks of accum)

  which equals Resolve over the union of all ranks' chains.

This module only moves numbers between ranks (all-reduce) and marshals them:
the sums come from the library and go back to it."""
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


def agree_p_sum(p_sum, n, group=None, device=None):
    """The ranks' initial-sample sums of p (FP64) and counts (int64), summed
    over ranks.  ``device`` holds the exchanged tensors (a CUDA device under
    NCCL; None means the CPU, for gloo)."""
    import torch
    s = torch.tensor([float(p_sum)], dtype=torch.float64, device=device)
    c = torch.tensor([int(n)], dtype=torch.int64, device=device)
    _all_reduce_sum(s, group)
    _all_reduce_sum(c, group)
    return float(s.item()), int(c.item())


def init_chains_agreed(r, n_chains, seed, params, group=None, device=None, frame=0):
    """Alg. 1 on every rank with one k0 for all ranks.  ``r`` is a renderer
    (``init_chains(n, seed, params, frame)``, ``p_sum()`` and
    ``k0_from_p_sum(p_sum, n, params)``).  When ``params.k0`` > 0 it is used
    as given; otherwise each rank first initialises with its own estimate,
    the ranks pool their initial samples' sums, and every rank initialises
    again with the k0 of the pooled samples given explicitly (the same seed
    draws the same samples, so only the clock sees the new k0).  Returns
    k0."""
    if params.k0 > 0:
        r.init_chains(n_chains, seed, params, frame)
        return float(params.k0)
    r.init_chains(n_chains, seed, params, frame)
    p_sum, n = agree_p_sum(*r.p_sum(), group=group, device=device)
    agreed = type(params).from_buffer_copy(params)
    agreed.k0 = r.k0_from_p_sum(p_sum, n, params)
    r.init_chains(n_chains, seed, agreed, frame)
    return float(agreed.k0)


def merge_and_resolve(accum, tour_count, k0, resolve, group=None):
    """accum: FP64 torch tensor (any device the process group supports),
    summed in place over ranks; the tour counts are summed as 64-bit
    integers.  ``resolve(accum, total_tour_count, k0)`` is the library's
    Resolve on the merged buffer (``renderer.resolve_accum``).  k0 is the
    one all ranks used (see init_chains_agreed).  Returns (image, total
    tour count)."""
    import torch
    tc = torch.tensor([int(tour_count)], dtype=torch.int64, device=accum.device)
    _all_reduce_sum(accum, group)
    _all_reduce_sum(tc, group)
    total = int(tc.item())
    return resolve(accum, total, float(k0)), total
