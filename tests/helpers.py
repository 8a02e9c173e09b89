"""Shared helpers for the GPU parity tests (inputs from the seeded
generators; expected values from the CPU oracle only)."""
from __future__ import annotations

import numpy as np

from oracle import oracle as o
from paper_2509_12232_gb300 import synth

# Per-pose bar: |E32 - E64| <= max(1e-3, 1e-4 |E64|) (1e-4 relative or 1e-3 absolute).
REL_TOL, ABS_TOL = 1e-4, 1e-3
# Poses whose oracle geometry lies within this distance (A) of a discontinuity
# of the score (the grid-box faces, the 8 A pair cutoff) are compared only for
# being one of the two branch values: FP32 and FP64 coordinates differ by
# ~1e-5 A and may fall on opposite sides.
MARGIN = 2e-4

PARAMS = synth.TYPE_PARAMS


def within(gpu, ref, rel=REL_TOL, abs_=ABS_TOL):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(gpu - ref) <= np.maximum(abs_, rel * np.abs(ref))


def gpu_pocket(dock, pk):
    return dock.dock_create_pocket(pk.x, pk.y, pk.z, pk.q, pk.type, pk.center, pk.radius, pk.spacing,
                                   PARAMS)


def gpu_ligands(dock, pocket, ligs):
    return dock.dock_load_ligands(pocket, ligs.atom_off, ligs.x, ligs.y, ligs.z, ligs.q, ligs.type,
                                  ligs.parent, ligs.tors_off, ligs.tors_b, ligs.ligand_id)


class OracleSide:
    """Oracle objects for a (pocket, ligand set) pair."""

    def __init__(self, pk, ligs, grid=None):
        self.P = o.Params(PARAMS)
        self.pk = pk
        self.pks = o.pocket_from(pk)
        self.grid = grid if grid is not None else o.grid_build(self.pks, self.P)
        self.ligs = ligs
        self._lig = {}

    def lig(self, l):
        if l not in self._lig:
            self._lig[l] = o.Ligand(**self.ligs.ligand(l))
        return self._lig[l]

    def score(self, l, genos, want_xyz=False):
        return o.score_poses(self.lig(l), self.P, self.grid, self.pk.center, genos, want_xyz)


def compare_scores(gpu, ref, margin):
    """(n_checked, n_margin, worst_rel, failures) with margin poses allowed to
    differ by one outside-grid penalty or one cutoff step."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    ok = within(gpu, ref)
    near = margin < MARGIN
    fails = np.nonzero(~ok & ~near)[0]
    rel = np.abs(gpu - ref) / np.maximum(1.0, np.abs(ref))
    return int((~near).sum()), int(near.sum()), float(rel[~near].max() if (~near).any() else 0), fails
