"""Shared helpers for the GPU parity tests (inputs from the seeded
generators; expected values from the CPU oracle only)."""
from __future__ import annotations

import numpy as np

from oracle import oracle as o
from paper_2509_12232_gb300 import synth

# Per-pose bar: |E32 - E64| <= max(1e-3, 1e-4 |E64|) (1e-4 relative or 1e-3 absolute).
REL_TOL, ABS_TOL = 1e-4, 1e-3
# Poses whose oracle geometry lies within this distance (A) of a discontinuity
# of the score (the grid-box faces, the 8 A pair cutoff) are compared with
# both branch values: FP32 and FP64 coordinates differ by ~1e-5 A, so an atom
# within the margin of a face may be inside on one side and outside (E_out)
# on the other, and a pair within the margin of 8 A may be counted on one
# side only. branch_jumps lists, per such atom or pair, the change of the
# oracle's score if it fell on the other side; a near pose passes when the
# GPU score is within the bar of the oracle's score plus some subset of them.
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


def _pair_jump(P, ti, tj, qi, qj, r):
    """Change of the score if a pair at r (within MARGIN of 8 A) fell on the
    other side of the cutoff: minus its term if counted, plus the term at
    8 A from below if not."""
    e = o.pair_terms(P, int(ti), int(tj), float(qi), float(qj), min(r, 8.0 - 1e-12))[3]
    return -e if r < 8.0 else e


def _atom_value(grid, T, t, q, x):
    vm = o.trilinear(grid, int(t), *x)
    ve = o.trilinear(grid, T, *x)
    vd = o.trilinear(grid, T + 1, *x)
    return vm + q * ve + abs(q) * vd


def branch_jumps(side, l, geno):
    """Score changes of the grid form's near-discontinuity items of one pose
    (oracle FP64 geometry): atoms within MARGIN of a box face and intra pairs
    within MARGIN of the cutoff."""
    lig = side.lig(l)
    g = side.grid
    T = side.P.n_types
    xyz = o.pose(lig, geno, side.pk.center)
    lo = g.origin
    hi = g.origin + (np.array(g.n) - 1) * g.h
    types, qs = lig.a["type"], lig.a["q"].astype(np.float64)
    jumps = []
    for a in range(lig.n):
        x = xyz[a]
        if np.all(x >= lo) and np.all(x <= hi):
            if min(np.min(x - lo), np.min(hi - x)) < MARGIN:
                jumps.append(o.EOUT - _atom_value(g, T, types[a], qs[a], x))
        else:
            xc = np.clip(x, lo, hi)
            if np.max(np.abs(x - xc)) < MARGIN:
                jumps.append(_atom_value(g, T, types[a], qs[a], xc) - o.EOUT)
    jumps += _intra_jumps(lig, side.P, xyz)
    return jumps


def _intra_jumps(lig, P, xyz):
    out = []
    pairs = o.topology(lig)[1]
    if len(pairs):
        r = np.linalg.norm(xyz[pairs[:, 0]] - xyz[pairs[:, 1]], axis=1)
        types, qs = lig.a["type"], lig.a["q"]
        for (i, j), ri in zip(pairs, r):
            if abs(ri - 8.0) < MARGIN:
                out.append(_pair_jump(P, types[i], types[j], qs[i], qs[j], ri))
    return out


def pairwise_jumps(lig, P, pks, xyz):
    """As branch_jumps for the pairwise form: intra pairs and ligand-protein
    pairs within MARGIN of the cutoff (no grid box)."""
    out = _intra_jumps(lig, P, xyz)
    prot = np.stack([pks.a["x"], pks.a["y"], pks.a["z"]], 1).astype(np.float64)
    d = np.linalg.norm(xyz[:, None, :] - prot[None], axis=2)
    for a, j in zip(*np.nonzero(np.abs(d - 8.0) < MARGIN)):
        out.append(_pair_jump(P, lig.a["type"][a], pks.a["type"][j], lig.a["q"][a],
                              pks.a["q"][j], d[a, j]))
    return out


def branch_ok(gpu, ref, jumps, rel=REL_TOL, abs_=ABS_TOL):
    """Whether gpu is within the bar of ref plus the sum of some subset of
    jumps (all subsets up to ten items; beyond, within the sum of their
    magnitudes)."""
    jumps = list(jumps)
    if len(jumps) > 10:
        return abs(gpu - ref) <= sum(abs(j) for j in jumps) + max(abs_, rel * abs(ref))
    for m in range(1 << len(jumps)):
        alt = ref + sum(j for b, j in enumerate(jumps) if m >> b & 1)
        if abs(gpu - alt) <= max(abs_, rel * abs(alt)):
            return True
    return False


def near_ok_grid(side, l, genos, got, ref, ok, near, **bar):
    """ok, with each margin pose that misses the bar re-checked against its
    branch values (grid form; bar: rel / abs_ of `within`)."""
    ok = np.array(ok, bool)
    for i in np.nonzero(~ok & np.asarray(near))[0]:
        ok[i] = branch_ok(float(got[i]), float(ref[i]), branch_jumps(side, l, genos[i]), **bar)
    return ok


def compare_scores(gpu, ref, margin, jumps_of):
    """(n_checked, n_margin, worst_rel, failures). Poses off the margin must
    meet the bar; a margin pose i must meet it against one of its branch
    values, jumps_of(i) giving the items' score changes (branch_jumps or
    pairwise_jumps)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    ok = within(gpu, ref)
    near = np.asarray(margin) < MARGIN
    for i in np.nonzero(near & ~ok)[0]:
        ok[i] = branch_ok(gpu[i], ref[i], jumps_of(int(i)))
    fails = np.nonzero(~ok)[0]
    rel = np.abs(gpu - ref) / np.maximum(1.0, np.abs(ref))
    return int((~near).sum()), int(near.sum()), float(rel[~near].max() if (~near).any() else 0), fails
