"""Distributing the batches of one system over several processes.

The paper parallelises every method across processes first ("Meeting the
Exascale Challenges": the code is built around distributed memory, with
shared memory and accelerators inside each process).  For grid integration
the batches are independent: each process integrates its own batches into
a partial H over the full sparsity pattern, one sum over processes gives H,
and each process owns the density of its own points.  The number of
electrons is the sum of the per-process traces.

This module holds the host logic of that split: a cost-balanced partition
of the batch list into contiguous ranges (batches from the recursive
bisection are spatially ordered, so a contiguous range keeps H locality)
and the one collective.  Any process group works (NCCL on GPUs, gloo on
CPU).
"""
from __future__ import annotations

import numpy as np


def batch_cost(points, n_active_fns):
    """Cost of each batch's contractions, P_b n_b^2 (at least 1)."""
    p = np.asarray(points, dtype=np.float64)
    n = np.asarray(n_active_fns, dtype=np.float64)
    return np.maximum(p * n * n, 1.0)


def partition_by_cost(cost, world: int):
    """Split batches 0..len(cost)-1 into `world` contiguous ranges of about
    equal total cost.  Batch k goes to the rank whose share of the total
    holds the midpoint of k's cost interval, so every batch lands exactly
    once, ranges keep the batch order, and no rank exceeds its share by more
    than one batch's cost.  Returns a list of index arrays (some may be
    empty when there are fewer batches than ranks)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    c = np.asarray(cost, dtype=np.float64)
    if c.ndim != 1 or np.any(~np.isfinite(c)) or np.any(c < 0):
        raise ValueError("cost must be a 1-D array of finite non-negative values")
    if len(c) == 0:
        return [np.zeros(0, np.int64) for _ in range(world)]
    hi = np.cumsum(c)
    total = hi[-1]
    if total <= 0:
        owner = (np.arange(len(c)) * world) // len(c)
    else:
        mid = hi - 0.5 * c
        owner = np.minimum((mid * world / total).astype(np.int64), world - 1)
    return [np.nonzero(owner == r)[0].astype(np.int64) for r in range(world)]


def allreduce_sum(t, group=None):
    """The one collective of the split H: elementwise FP64 sum over ranks."""
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
