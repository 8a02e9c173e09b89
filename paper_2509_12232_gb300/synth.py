"""Seeded synthetic inputs for the docking hot path.

This module only draws inputs: protein pockets, ligands and the atom-type
parameter table. It computes no energy, pose or search step, so both the CUDA
library and the CPU oracle can be fed from it without sharing any of the
method's arithmetic.

The paper's datasets (a ~2,500-molecule MEDIATE subset and the PDBbind complex
1a30, Section VII "Dataset") are not available; these generators stand in for
them with the workload shapes of the five synthetic configurations:

* ``c1`` one 24-atom ligand with 4 rotatable bonds; 1,500-atom pocket, 12 A.
* ``c2`` 1,000 ligands, 10-60 atoms, 0-12 torsions; 4,000-atom pocket, 16 A.
* ``c3`` 100,000 ligands, lognormal size (mean 30, sd 10, 8-100 atoms),
  Poisson(5) torsions clipped at 16; 4,000-atom pocket.
* ``c5`` 1,000,000 ligands with the c2 size mix; 10,000-atom pocket, 20 A.

Pocket reading: N atoms at >= 2.8 A spacing cannot fit inside a sphere of the
stated radius (packing fraction 2.4-3.4), so the radius is the empty binding
cavity and the atoms are dart-thrown into the shell around it, out to the
radius where the shell's packing fraction is 0.25.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Atom-type parameter table (input data).
#
# Seven heavy-atom types.  Values are modelled on the AutoDock4 force field's
# published per-type parameters (Morris et al. 2009, the paper's AutoDock4
# citation): Rii is the vdW well distance for a like pair, eps the well depth,
# vol the atomic fragmental volume and solpar the atomic solvation parameter.
# "ND" is a heavy-atom hydrogen-bond donor pseudo-type, needed because the
# ligands carry no hydrogens; hb_R / hb_eps give the 12-10 well of a
# donor-acceptor pair, taken from the acceptor.
# ---------------------------------------------------------------------------
TYPE_NAMES = ("C", "A", "N", "NA", "OA", "SA", "ND")
HB_NONE, HB_DONOR, HB_ACCEPTOR = 0, 1, 2

TYPE_PARAMS = {
    "Rii":     np.array([4.00, 4.00, 3.50, 3.50, 3.20, 4.00, 3.50], np.float32),
    "eps":     np.array([0.150, 0.150, 0.160, 0.160, 0.200, 0.200, 0.160], np.float32),
    "vol":     np.array([33.51, 33.51, 22.45, 22.45, 17.16, 33.51, 22.45], np.float32),
    "solpar":  np.array([-0.00143, -0.00052, -0.00162, -0.00162, -0.00251, -0.00214,
                         -0.00162], np.float32),
    "hb_role": np.array([0, 0, 0, 2, 2, 2, 1], np.int32),
    "hb_R":    np.array([0.0, 0.0, 0.0, 2.9, 2.8, 3.3, 0.0], np.float32),
    "hb_eps":  np.array([0.0, 0.0, 0.0, 5.0, 5.0, 1.0, 0.0], np.float32),
}
N_TYPES = len(TYPE_NAMES)


@dataclass
class Pocket:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    q: np.ndarray
    type: np.ndarray
    center: tuple
    radius: float
    spacing: float = 0.375

    @property
    def n_atoms(self) -> int:
        return int(self.x.shape[0])


@dataclass
class LigandSet:
    """Ligands in CSR form.

    Atoms of ligand l are ``atom_off[l]:atom_off[l+1]``; within a ligand the
    atoms are in topological order (``parent[i] < i``, atom 0 is the root with
    parent -1; parents are ligand-local indices).  The rotatable bonds of
    ligand l are ``tors_b[tors_off[l]:tors_off[l+1]]``: bond (parent[b], b),
    listed in increasing b, so an ancestor bond comes before its descendants.
    """
    atom_off: np.ndarray
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    q: np.ndarray
    type: np.ndarray
    parent: np.ndarray
    tors_off: np.ndarray
    tors_b: np.ndarray
    ligand_id: np.ndarray = field(default=None)

    @property
    def n_ligands(self) -> int:
        return int(self.atom_off.shape[0] - 1)

    def n_atoms(self, l: int) -> int:
        return int(self.atom_off[l + 1] - self.atom_off[l])

    def n_tors(self, l: int) -> int:
        return int(self.tors_off[l + 1] - self.tors_off[l])

    def subset(self, idx) -> "LigandSet":
        """A new LigandSet holding ligands ``idx`` (in that order)."""
        idx = np.asarray(idx, np.int64)
        na = np.diff(self.atom_off)[idx]
        nt = np.diff(self.tors_off)[idx]
        atoms = np.concatenate([np.arange(self.atom_off[i], self.atom_off[i + 1]) for i in idx]) \
            if len(idx) else np.zeros(0, np.int64)
        tors = np.concatenate([np.arange(self.tors_off[i], self.tors_off[i + 1]) for i in idx]) \
            if len(idx) else np.zeros(0, np.int64)
        return LigandSet(
            atom_off=np.concatenate([[0], np.cumsum(na)]).astype(np.int32),
            x=self.x[atoms], y=self.y[atoms], z=self.z[atoms], q=self.q[atoms],
            type=self.type[atoms], parent=self.parent[atoms],
            tors_off=np.concatenate([[0], np.cumsum(nt)]).astype(np.int32),
            tors_b=self.tors_b[tors], ligand_id=self.ligand_id[idx].copy())

    def ligand(self, l: int) -> dict:
        a0, a1 = int(self.atom_off[l]), int(self.atom_off[l + 1])
        t0, t1 = int(self.tors_off[l]), int(self.tors_off[l + 1])
        return dict(x=self.x[a0:a1], y=self.y[a0:a1], z=self.z[a0:a1], q=self.q[a0:a1],
                    type=self.type[a0:a1], parent=self.parent[a0:a1],
                    tors_b=self.tors_b[t0:t1], ligand_id=int(self.ligand_id[l]))


# ---------------------------------------------------------------------------
# Pocket
# ---------------------------------------------------------------------------
def shell_outer_radius(n_atoms: int, radius: float, min_sep: float = 2.8,
                       packing: float = 0.25) -> float:
    """Outer radius of a shell around the cavity holding n hard spheres of
    diameter min_sep at the given packing fraction."""
    r_hs = 0.5 * min_sep
    return (radius ** 3 + n_atoms * r_hs ** 3 / packing) ** (1.0 / 3.0)


def make_pocket(n_atoms: int, radius: float, seed: int = 0, spacing: float = 0.375,
                min_sep: float = 2.8, packing: float = 0.25,
                center=(0.0, 0.0, 0.0)) -> Pocket:
    """Dart-throw n_atoms protein atoms (min spacing min_sep) into the shell
    radius <= |x - center| <= R_out; uniform types, charges N(0, 0.4)."""
    rng = np.random.Generator(np.random.Philox(seed))
    r_out = shell_outer_radius(n_atoms, radius, min_sep, packing)
    cell = min_sep
    grid: dict = {}
    pts = []
    tries = 0
    while len(pts) < n_atoms:
        m = 4096
        u = rng.random(m)
        r = (radius ** 3 + u * (r_out ** 3 - radius ** 3)) ** (1.0 / 3.0)
        d = rng.normal(size=(m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        cand = d * r[:, None]
        for p in cand:
            tries += 1
            key = tuple(np.floor(p / cell).astype(np.int64))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for q in grid.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                            if (p[0] - q[0]) ** 2 + (p[1] - q[1]) ** 2 + (p[2] - q[2]) ** 2 < min_sep ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                grid.setdefault(key, []).append(p)
                pts.append(p)
                if len(pts) == n_atoms:
                    break
        if tries > 200 * n_atoms:
            raise RuntimeError("pocket dart throwing did not converge")
    xyz = np.array(pts, np.float64) + np.asarray(center, np.float64)[None, :]
    types = rng.integers(0, N_TYPES, size=n_atoms).astype(np.uint8)
    q = rng.normal(0.0, 0.4, size=n_atoms)
    return Pocket(x=xyz[:, 0].astype(np.float32), y=xyz[:, 1].astype(np.float32),
                  z=xyz[:, 2].astype(np.float32), q=q.astype(np.float32), type=types,
                  center=tuple(float(c) for c in center), radius=float(radius),
                  spacing=float(spacing))


# ---------------------------------------------------------------------------
# Ligands
# ---------------------------------------------------------------------------
def make_ligands(rng: np.random.Generator, n_atoms, n_tors_req, id_base: int = 0,
                 bond=(1.45, 1.55), min_nonbonded: float = 2.0) -> LigandSet:
    """Random-tree ligands, vectorised over ligands.

    Atom i (i >= 1) attaches to a random earlier atom with fewer than four
    bonds, at a bond length uniform in ``bond`` and a uniform direction, and is
    kept only if it is at least ``min_nonbonded`` from every other atom.
    Rotatable bonds are drawn from the bonds (parent[b], b) that leave at least
    two atoms on each side; charges N(0, 0.3) shifted to sum to zero; types
    uniform over the seven types.
    """
    n_atoms = np.asarray(n_atoms, np.int64)
    n_tors_req = np.asarray(n_tors_req, np.int64)
    L = n_atoms.shape[0]
    nmax = int(n_atoms.max()) if L else 0
    pos = np.zeros((L, max(nmax, 1), 3), np.float64)
    parent = np.full((L, max(nmax, 1)), -1, np.int64)
    deg = np.zeros((L, max(nmax, 1)), np.int64)
    for i in range(1, nmax):
        pend = np.nonzero(n_atoms > i)[0]
        for attempt in range(400):
            if pend.size == 0:
                break
            m = pend.size
            w = rng.random((m, i))
            w[deg[pend, :i] >= 4] = -1.0
            p = np.argmax(w, axis=1)
            d = rng.normal(size=(m, 3))
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            blen = rng.uniform(bond[0], bond[1], size=m)
            x = pos[pend, p] + d * blen[:, None]
            dist = np.linalg.norm(pos[pend, :i] - x[:, None, :], axis=2)
            dist[np.arange(m), p] = np.inf
            ok = np.all(dist >= min_nonbonded, axis=1)
            acc = pend[ok]
            pos[acc, i] = x[ok]
            parent[acc, i] = p[ok]
            deg[acc, p[ok]] += 1
            deg[acc, i] = 1
            pend = pend[~ok]
        if pend.size:
            raise RuntimeError("ligand growth did not converge")

    xs, ys, zs, qs, ts, ps, tb = [], [], [], [], [], [], []
    tcount = np.zeros(L, np.int64)
    for l in range(L):
        n = int(n_atoms[l])
        par = parent[l, :n]
        # subtree sizes (children have larger indices than parents)
        size = np.ones(n, np.int64)
        for a in range(n - 1, 0, -1):
            size[par[a]] += size[a]
        elig = np.array([b for b in range(1, n) if size[b] >= 2 and n - size[b] >= 2], np.int64)
        k = int(min(n_tors_req[l], elig.size))
        chosen = np.sort(rng.choice(elig, size=k, replace=False)) if k else np.zeros(0, np.int64)
        q = rng.normal(0.0, 0.3, size=n)
        q = q - q.mean()
        typ = rng.integers(0, N_TYPES, size=n)
        xs.append(pos[l, :n, 0]); ys.append(pos[l, :n, 1]); zs.append(pos[l, :n, 2])
        qs.append(q); ts.append(typ); ps.append(par); tb.append(chosen)
        tcount[l] = k
    cat = (lambda a, dt: np.concatenate(a).astype(dt) if a else np.zeros(0, dt))
    return LigandSet(
        atom_off=np.concatenate([[0], np.cumsum(n_atoms)]).astype(np.int32),
        x=cat(xs, np.float32), y=cat(ys, np.float32), z=cat(zs, np.float32),
        q=cat(qs, np.float32), type=cat(ts, np.uint8), parent=cat(ps, np.int16),
        tors_off=np.concatenate([[0], np.cumsum(tcount)]).astype(np.int32),
        tors_b=cat(tb, np.int16),
        ligand_id=(np.arange(L, dtype=np.uint64) + np.uint64(id_base)))


# ---------------------------------------------------------------------------
# The five workload configurations
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    pocket_atoms: int
    radius: float
    n_ligands: int
    pop: int
    generations: int
    sizes: str          # "fixed24", "uniform", "lognormal"


WORKLOADS = {
    "c1": Workload("c1", 1500, 12.0, 1, 256, 10, "fixed24"),
    "c2": Workload("c2", 4000, 16.0, 1000, 1024, 50, "uniform"),
    "c3": Workload("c3", 4000, 16.0, 100_000, 512, 30, "lognormal"),
    "c5": Workload("c5", 10_000, 20.0, 1_000_000, 2048, 40, "uniform"),
}


def ligand_sizes(rng: np.random.Generator, kind: str, n: int):
    if kind == "fixed24":
        return np.full(n, 24, np.int64), np.full(n, 4, np.int64)
    if kind == "uniform":
        return rng.integers(10, 61, size=n), rng.integers(0, 13, size=n)
    if kind == "lognormal":
        sigma = math.sqrt(math.log(1.0 + (10.0 / 30.0) ** 2))
        mu = math.log(30.0) - 0.5 * sigma * sigma
        na = np.clip(np.rint(rng.lognormal(mu, sigma, size=n)), 8, 100).astype(np.int64)
        nt = np.minimum(rng.poisson(5.0, size=n), 16)
        return na, nt
    raise ValueError(kind)


def make_workload(name: str, n_ligands: int | None = None, seed: int = 0,
                  pocket: bool = True):
    """(pocket, ligands, workload) for one configuration.

    The pocket uses ``seed``; the ligand set is drawn from a Philox stream
    keyed by ``seed + 1000``.  ``n_ligands`` truncates the set (the first n
    ligands of the full draw order are the same for any n only for the sizes;
    geometry is drawn per call).
    """
    w = WORKLOADS[name]
    n = w.n_ligands if n_ligands is None else int(n_ligands)
    pk = make_pocket(w.pocket_atoms, w.radius, seed=seed) if pocket else None
    rng = np.random.Generator(np.random.Philox(seed + 1000))
    na, nt = ligand_sizes(rng, w.sizes, n)
    ligs = make_ligands(rng, na, nt)
    return pk, ligs, w


SCREEN_CHUNK = 50_000


def screen_chunk(name: str, c: int, size: int = SCREEN_CHUNK, seed: int = 0) -> LigandSet:
    """Ligands [c size, (c + 1) size) of a large screen (``c5``: 20 chunks of
    50,000), drawn from their own Philox stream keyed by (seed + 1000, c) so
    any chunk can be made alone and in parallel; ligand ids c size + i."""
    w = WORKLOADS[name]
    n = max(0, min(size, w.n_ligands - c * size))
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed + 1000, c])))
    na, nt = ligand_sizes(rng, w.sizes, n)
    return make_ligands(rng, na, nt, id_base=c * size)


def screen_chunks(name: str, size: int = SCREEN_CHUNK) -> int:
    """Number of chunks of the screen `name` at `size` ligands per chunk."""
    return -(-WORKLOADS[name].n_ligands // size)
