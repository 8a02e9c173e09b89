"""Ligand sharding across GPUs (one process per GPU).

Ligands are independent (the paper's node-level parallelism is one ligand per
worker, Section IV), so a batch splits into contiguous ranges, one per rank,
balanced by estimated cost; no collective touches the data path.
"""
from __future__ import annotations

import numpy as np


def ligand_costs(atom_off, tors_off) -> np.ndarray:
    """Per-ligand cost estimate of the search: pairs ~ n^2 / 2, plus atoms and torsions."""
    n = np.diff(np.asarray(atom_off, np.int64)).astype(np.float64)
    k = np.diff(np.asarray(tors_off, np.int64)).astype(np.float64)
    return 0.5 * n * (n - 1) + 6.0 * n + 12.0 * k + 60.0


def balanced_ranges(costs, world: int):
    """Split indices 0..len(costs) into `world` contiguous ranges whose cost
    sums are as even as the prefix sums allow: range r ends at the first
    index whose prefix cost reaches (r + 1) / world of the total."""
    c = np.asarray(costs, np.float64)
    n = c.shape[0]
    if world < 1:
        raise ValueError("world must be >= 1")
    pref = np.concatenate([[0.0], np.cumsum(c)])
    total = pref[-1]
    bounds = [0]
    for r in range(1, world):
        b = int(np.searchsorted(pref, total * r / world, side="left"))
        bounds.append(min(max(b, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def gather_records(records: np.ndarray, group=None) -> np.ndarray:
    """The one exchange of a sharded run: every rank's per-ligand records (a
    structured numpy array, e.g. dock_result rows of its range) gathered in
    rank order, so the result lists the records in global ligand order when
    the ranges are balanced_ranges'. Host-side, over torch.distributed (gloo
    or any backend that moves CPU tensors); returns the gathered array on
    every rank."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rec = np.ascontiguousarray(records)
    raw = torch.from_numpy(rec.view(np.uint8).reshape(-1).copy())
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([raw.numel()], dtype=torch.int64), group=group)
    m = max(int(s.item()) for s in sizes)
    pad = torch.zeros(max(m, 1), dtype=torch.uint8)
    pad[:raw.numel()] = raw
    got = [torch.zeros(max(m, 1), dtype=torch.uint8) for _ in range(world)]
    dist.all_gather(got, pad, group=group)
    parts = [g[:int(s.item())].numpy() for g, s in zip(got, sizes)]
    return np.concatenate(parts).view(rec.dtype) if parts else rec[:0]
