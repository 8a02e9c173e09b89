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
