"""Schedule autotuner for the Restore step.

Chooses, by timing short runs on the caller's workload through the public
API, the launch schedule that the hot path leaves open:

* ``traverse_blocks`` - resident blocks per SM of the persistent traversal
  pass (chains in flight per SM; 0 = every block that fits),
* ``refill`` - the busy-lane count below which a traversal warp fetches new
  rays,
* ``steps_per_frame`` - Restore steps per captured CUDA-graph frame (steps per
  launch of the graph),
* ``tail_bounce`` - the bounce from whose shading on each path finishes in
  one persistent pass (0: every bounce as its own launches).

The traversal stack depth is fixed at build time (48 entries for the flat
hierarchies, 64 for the two-level walk; checked against every BVH at upload),
so it is not a run-time choice.
"""
from __future__ import annotations

import itertools

import torch


def default_candidates():
    return [dict(traverse_blocks=b, refill=f, steps_per_frame=F, tail_bounce=t)
            for b, f, F, t in itertools.product((0, 6), (12, 16, 20), (2, 4), (0, 4, 6))]


def apply(r, cand):
    r.set_option("traverse_blocks", cand["traverse_blocks"])
    r.set_option("refill", cand["refill"])
    r.set_option("tail_bounce", cand["tail_bounce"])


def autotune(r, stream, n_chains, seed, params, candidates=None, steps=8, reps=2):
    """Times ``steps`` Restore steps (after init and one captured frame) for
    each candidate schedule on renderer ``r`` (created on ``stream``) and
    applies the fastest.  Returns (best candidate, [(ms per step, candidate)])."""
    candidates = candidates or default_candidates()
    results = []
    for cand in candidates:
        apply(r, cand)
        F = cand["steps_per_frame"]
        n_frames = max(1, steps // F)
        r.init_chains(n_chains, seed, params)
        r.frame(F)  # capture
        stream.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n_frames):
                r.frame(F)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / (n_frames * F))
        results.append((best, cand))
    ms, cand = min(results, key=lambda t: t[0])
    apply(r, cand)
    return cand, results
