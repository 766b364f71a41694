"""Several GPUs, one process each: the batched form shards its clouds.

Clouds are independent, so a batch splits across ranks with no exchange on
the data path: clouds sorted by decreasing size are dealt round robin (a
greedy balance of the quadratic per-cloud work), each rank computes its share
with one batched call on its own GPU, and the pairs are gathered on the host.
A single cloud does not shard (its sort and reduction are global): several
GPUs only run replicas of it.
"""
from __future__ import annotations

import numpy as np


def shard_clouds(sizes, world: int, rank: int):
    """Indices of the clouds rank `rank` computes: decreasing size, dealt round robin."""
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    return order[rank::world]


def local_batch(points, offsets, idx):
    """Points (numpy) and offsets of the clouds `idx`, packed back to back."""
    offsets = np.asarray(offsets, dtype=np.int64)
    parts = [points[offsets[i]:offsets[i + 1]] for i in idx]
    offs = np.zeros(len(idx) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([p.shape[0] for p in parts])
    pts = np.concatenate(parts, 0) if parts else np.zeros((0, points.shape[1]), points.dtype)
    return np.ascontiguousarray(pts), offs


def sharded_batched(points, offsets, dmax=1, threshold=float("inf"), group=None, compute=None):
    """Barcodes of every cloud, computed across the ranks of `group`.

    Returns, on every rank, a list over clouds of per-dimension pair arrays.
    `compute(pts, offs, dmax, threshold)` returns that list for a packed local
    batch; by default it is one vr_barcodes_batched call on this rank's GPU."""
    import torch.distributed as dist
    world = dist.get_world_size(group) if group is not None or dist.is_initialized() else 1
    rank = dist.get_rank(group) if world > 1 else 0
    offsets = np.asarray(offsets, dtype=np.int64)
    sizes = np.diff(offsets)
    idx = shard_clouds(sizes, world, rank)
    pts, offs = local_batch(points, offsets, idx)
    if compute is None:
        from . import vr

        def compute(p, o, d, t):
            bb = vr.barcodes_batched(p, o, dmax=d, threshold=t)
            return [[bb.cloud(i, q) for q in range(d + 1)] for i in range(len(o) - 1)]
    local = compute(pts, offs, dmax, threshold) if len(idx) else []
    if world == 1:
        return local
    gathered = [None] * world
    dist.all_gather_object(gathered, (idx, local), group=group)
    out = [None] * len(sizes)
    for ids, res in gathered:
        for i, r in zip(ids, res):
            out[i] = r
    return out
