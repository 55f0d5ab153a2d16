"""Sharding a trace over ranks and merging the ranks' outputs.

Every ray is keyed by (global segment index, bunch index) through the
counter-based generator, so ranks trace disjoint contiguous segment ranges
(seg_base = start of the range) and exchange nothing while tracing.  After
tracing, the per-(shower, telescope) counts are summed, the photon sums are
summed, and the hit lists, each sorted by (shower, telescope, segment,
bunch), are concatenated in rank order and stably re-sorted by
(shower, telescope): segment indices grow with the rank, so that yields the
single-process order.  When the ranges are cut at shower boundaries every
(shower, telescope) group lives on one rank and the merged sums equal the
single-process ones bit for bit; otherwise they agree to rounding.
"""
from __future__ import annotations

import numpy as np


def plan(n_segs: int, world: int, shower: np.ndarray | None = None) -> list[tuple[int, int]]:
    """Contiguous [lo, hi) segment ranges, one per rank, balanced by segment count.

    With `shower` (non-decreasing shower id per segment) cuts fall only on
    shower boundaries, so no (shower, telescope) group is split."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if shower is None:
        edges = [(n_segs * r) // world for r in range(world + 1)]
    else:
        shower = np.asarray(shower)
        if len(shower) != n_segs:
            raise ValueError("shower ids must have one entry per segment")
        if n_segs and np.any(np.diff(shower.astype(np.int64)) < 0):
            raise ValueError("segments must be grouped by shower in non-decreasing order")
        starts = np.flatnonzero(np.r_[True, shower[1:] != shower[:-1]]) if n_segs else np.zeros(0, np.int64)
        bounds = np.r_[starts, n_segs]
        edges = [0]
        for r in range(1, world):
            target = (n_segs * r) // world
            j = int(np.searchsorted(bounds, target))
            # nearest shower boundary to the balanced cut, never moving backwards
            if j > 0 and (j == len(bounds) or target - bounds[j - 1] <= bounds[j] - target):
                j -= 1
            edges.append(max(edges[-1], int(bounds[min(j, len(bounds) - 1)])))
        edges.append(n_segs)
    return [(edges[r], edges[r + 1]) for r in range(world)]


def merge_hits(parts: list[np.ndarray], group_of) -> np.ndarray:
    """Concatenate rank-ordered, individually sorted hit lists and restore the global order.

    `group_of(hits)` returns the (shower * n_tel + telescope) group of each hit."""
    parts = [p for p in parts if len(p)]
    if not parts:
        return np.zeros(0, dtype=parts[0].dtype) if parts else np.zeros(0)
    m = np.concatenate(parts)
    return m[np.argsort(group_of(m), kind="stable")]


def allgather_records(arr: np.ndarray, device="cpu", group=None) -> list[np.ndarray]:
    """Every rank's structured array, in rank order (torch.distributed, any backend)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    raw = np.ascontiguousarray(arr).view(np.uint8).reshape(-1)
    n = torch.tensor([raw.size], dtype=torch.int64, device=device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(max(sizes), 1)
    buf = torch.zeros(cap, dtype=torch.uint8, device=device)
    if raw.size:
        buf[: raw.size] = torch.from_numpy(raw).to(device)
    outs = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    return [o[:s].cpu().numpy().view(arr.dtype).copy() for o, s in zip(outs, sizes)]


def reduce_totals(counts: np.ndarray, sums: np.ndarray, device="cpu", group=None):
    """Sum the per-group counts (int64) and photon sums (FP64) over ranks."""
    import torch
    import torch.distributed as dist
    c = torch.from_numpy(np.ascontiguousarray(counts, dtype=np.int64)).to(device)
    s = torch.from_numpy(np.ascontiguousarray(sums, dtype=np.float64)).to(device)
    dist.all_reduce(c, group=group)
    dist.all_reduce(s, group=group)
    return c.cpu().numpy().reshape(counts.shape), s.cpu().numpy().reshape(sums.shape)


def merge(hits: np.ndarray, counts: np.ndarray, sums: np.ndarray, group_of, device="cpu", group=None):
    """The single-process (hits, counts, sums) from each rank's shard output."""
    parts = allgather_records(hits, device=device, group=group)
    c, s = reduce_totals(counts, sums, device=device, group=group)
    return merge_hits(parts, group_of), c, s
