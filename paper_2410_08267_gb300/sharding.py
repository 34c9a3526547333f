"""Host-side multi-GPU logic: one process per GPU, no data-path collective.

Every trajectory and every radius of the method is independent (Sec. II.C,
Eq. localdensity: each n/nbar(x0) is its own quadrature), so a batch of
requests partitions across ranks with nothing exchanged while the kernels run.
This module holds the three host steps of that scheme:

* ``partition``: assign whole requests to ranks, balancing their
  trajectory-steps (longest-processing-time greedy; deterministic, so every
  rank computes the same assignment without communicating);
* ``max_over_ranks``: the slowest rank's time (the job's time);
* ``gather_profiles``: collect each rank's n/nbar arrays on every rank, in
  request order, after all kernels have finished.

The process group may be NCCL (GPU tensors) or gloo (CPU tensors); the
functions take the device of the reduction tensor from the backend.
"""
from __future__ import annotations

import heapq
from typing import Dict, List, Sequence

import numpy as np


def partition(weights: Sequence[float], world: int) -> List[List[int]]:
    """Split items with the given costs over ``world`` ranks.

    Items are taken in decreasing cost (ties by index) and each goes to the
    rank with the smallest load so far (ties by rank).  Returns, per rank,
    the ascending list of item indices.  Every index appears exactly once.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    w = [float(x) for x in weights]
    if any(x < 0 or not np.isfinite(x) for x in w):
        raise ValueError("weights must be finite and non-negative")
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    heap = [(0.0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + w[i], r))
    return [sorted(x) for x in out]


def partition_problems(problems, world: int) -> List[List[int]]:
    """``partition`` of requests by their trajectory-steps."""
    return partition([pb.traj_steps for pb in problems], world)


def _device(dist):
    import torch
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def max_over_ranks(value: float, dist=None) -> float:
    """The largest ``value`` over all ranks (the value itself without a group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_profiles(local: Dict[int, np.ndarray], n_items: int, dist=None) -> List[np.ndarray]:
    """Collect per-request results computed on different ranks.

    ``local`` maps request index -> this rank's result array.  Returns the
    list of all ``n_items`` arrays in request order on every rank.  Raises if
    an index is missing or was computed twice.
    """
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        parts = [local]
    else:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, {int(k): np.asarray(v) for k, v in local.items()})
    out: List[np.ndarray] = [None] * n_items
    for part in parts:
        for k, v in part.items():
            if not 0 <= k < n_items:
                raise ValueError(f"request index {k} out of range")
            if out[k] is not None:
                raise ValueError(f"request {k} computed on two ranks")
            out[k] = v
    missing = [i for i, v in enumerate(out) if v is None]
    if missing:
        raise ValueError(f"requests {missing[:8]} computed on no rank")
    return out
