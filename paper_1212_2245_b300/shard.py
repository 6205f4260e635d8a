"""Sharding of independent images across ranks (one process per GPU).

Images of a batch are independent problems, so the forward pipeline shards
by image with no exchange at all: every rank deblurs its own images.  The
assignment is longest-processing-time first on the cost pixels x iterations
(Graham's LPT rule: sort by cost, give each image to the least loaded rank),
which keeps the largest rank load within 4/3 - 1/(3m) of the optimum for m
ranks.

The reverse mode (tuning taps, alpha and K on a batch) has one exchange
step: each rank's loss is the mean over its own images, the batch loss is
the image-count-weighted mean of the ranks' losses, so the parameter
gradient of the batch is the sum over ranks of n_r / n_total times the
rank's gradient: one all-reduce of kh*kw + 2 numbers.  The gradients with
respect to the images stay with the rank that owns the image.
"""
from __future__ import annotations

import heapq
from typing import Sequence

import torch
import torch.distributed as dist


def lpt_partition(costs: Sequence[float], n_ranks: int) -> list[list[int]]:
    """Indices of the images of each rank (each list ascending).  Ties in cost
    keep the original order; ties in load go to the lower rank."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(n_ranks)]
    parts: list[list[int]] = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def rank_images(costs: Sequence[float], n_ranks: int, rank: int) -> list[int]:
    return lpt_partition(costs, n_ranks)[rank]


def image_costs(shapes: Sequence[tuple[int, int]], iters: Sequence[int] | int) -> list[float]:
    """Pixels x iterations of each image."""
    its = [iters] * len(shapes) if isinstance(iters, int) else list(iters)
    return [float(h * w * max(k, 1)) for (h, w), k in zip(shapes, its)]


def combine_param_grads(grads: Sequence[torch.Tensor], n_local: int, n_total: int, group=None) -> None:
    """In place: turn each rank's gradients of its own mean loss into the
    gradients of the batch mean loss (scale by n_local / n_total, then sum
    over ranks).  Without an initialised process group (one rank) only the
    scaling applies."""
    if n_total <= 0:
        raise ValueError("n_total must be positive")
    flat = torch.cat([g.reshape(-1).to(torch.float64) for g in grads]) * (float(n_local) / float(n_total))
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for g in grads:
        n = g.numel()
        g.copy_(flat[off:off + n].reshape(g.shape).to(g.dtype))
        off += n
