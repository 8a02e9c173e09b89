"""ctypes front end of the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it. It imports nothing from the CUDA package
and takes plain numpy arrays, so inputs drawn by the shared seeded generators
can be fed to both sides.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "surrogate.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
# the FP32 auto-vectorised CPU baseline (simd_fp32.c) links the oracle's GA
_SRC32 = os.path.join(_HERE, "simd_fp32.c")
_LIB32 = os.path.join(_HERE, "libcpu32.so")

EMAX = 1.0e5
EOUT = 1000.0
CUTOFF = 8.0


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP64, -O2, no fast-math, no FP contraction)."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in srcs)
    if stale:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-pthread", "-o", tmp] + srcs + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def build_cpu32(force: bool = False) -> str:
    """Compile libcpu32.so: simd_fp32.c at -O3 -ffast-math -fopenmp-simd (the
    paper's auto-vectorised FP32 style) linked with oracle.c built as for
    liboracle.so (its GA and topology)."""
    srcs = [_SRC[0], _SRC32]
    stale = force or not os.path.exists(_LIB32) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB32) for s in srcs)
    if stale:
        pid = os.getpid()
        o1, o2 = _LIB32 + ".%d.oracle.o" % pid, _LIB32 + ".%d.simd.o" % pid
        tmp = _LIB32 + ".%d.tmp" % pid
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-ffp-contract=off",
                               "-fno-fast-math", "-pthread", "-c", _SRC[0], "-o", o1])
        subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fPIC", "-ffast-math", "-fopenmp-simd",
                               "-pthread", "-c", _SRC32, "-o", o2])
        subprocess.check_call(["gcc", "-shared", "-pthread", "-o", tmp, o1, o2, "-lm"])
        os.replace(tmp, _LIB32)
        for f in (o1, o2):
            os.unlink(f)
    return _LIB32


_lib = None
_lib32 = None


def lib32():
    global _lib32
    if _lib32 is None:
        L = C.CDLL(build_cpu32())
        L.cpu32_score_poses.restype = C.c_int
        L.cpu32_score_poses.argtypes = [C.POINTER(OrcLigand), C.POINTER(OrcParams), C.POINTER(OrcGrid),
                                        P_d, P_f, C.c_int, C.c_int64, P_f]
        L.cpu32_dock_batch.restype = None
        L.cpu32_dock_batch.argtypes = [C.POINTER(OrcBatch), C.POINTER(OrcParams), C.POINTER(OrcPocket),
                                       C.POINTER(OrcGrid), C.c_int, C.c_int, C.c_float, C.c_float,
                                       C.c_uint64, C.c_int, P_f, P_i32, P_f, P_f]
        _lib32 = L
    return _lib32


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


# ---------------------------------------------------------------------------
# C structs
# ---------------------------------------------------------------------------
P_f = C.POINTER(C.c_float)
P_d = C.POINTER(C.c_double)
P_u8 = C.POINTER(C.c_uint8)
P_i16 = C.POINTER(C.c_int16)
P_i32 = C.POINTER(C.c_int32)
P_u64 = C.POINTER(C.c_uint64)
P_i64 = C.POINTER(C.c_int64)


class OrcParams(C.Structure):
    _fields_ = [("n_types", C.c_int32), ("Rii", P_f), ("eps", P_f), ("vol", P_f),
                ("solpar", P_f), ("hb_R", P_f), ("hb_eps", P_f), ("hb_role", P_i32)]


class OrcLigand(C.Structure):
    _fields_ = [("n", C.c_int32), ("x", P_f), ("y", P_f), ("z", P_f), ("q", P_f),
                ("type", P_u8), ("parent", P_i16), ("k", C.c_int32), ("tors_b", P_i16)]


class OrcPocket(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("x", P_f), ("y", P_f), ("z", P_f), ("q", P_f),
                ("type", P_u8), ("center", C.c_double * 3), ("radius", C.c_double),
                ("spacing", C.c_double)]


class OrcGrid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("n_types", C.c_int32),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double), ("h", C.c_double),
                ("maps", P_d)]


class OrcLsParams(C.Structure):
    _fields_ = [("rate", C.c_float), ("max_its", C.c_int32), ("max_succ", C.c_int32),
                ("max_fail", C.c_int32), ("rho", C.c_float), ("rho_lb", C.c_float)]


class OrcSearch(C.Structure):
    _fields_ = [("pop", C.c_int32), ("generations", C.c_int32), ("p_cross", C.c_float),
                ("p_mut", C.c_float), ("seed", C.c_uint64), ("ls", OrcLsParams)]


# objective of a Solis-Wets probe: (genotype, iteration, 0 forward / 1 backward, ctx) -> score
LS_OBJECTIVE = C.CFUNCTYPE(C.c_float, C.POINTER(C.c_float), C.c_int32, C.c_int32, C.c_void_p)


class OrcBatch(C.Structure):
    _fields_ = [("n_ligands", C.c_int32), ("atom_off", P_i32), ("tors_off", P_i32),
                ("x", P_f), ("y", P_f), ("z", P_f), ("q", P_f), ("type", P_u8),
                ("parent", P_i16), ("tors_b", P_i16), ("ligand_id", P_u64)]


def _declare(L):
    L.orc_dielectric.restype = C.c_double
    L.orc_dielectric.argtypes = [C.c_double]
    L.orc_disp_raw.restype = C.c_double
    L.orc_disp_raw.argtypes = [C.POINTER(OrcParams), C.c_int, C.c_int, C.c_double]
    L.orc_pair_terms.restype = None
    L.orc_pair_terms.argtypes = [C.POINTER(OrcParams), C.c_int, C.c_int, C.c_double, C.c_double,
                                 C.c_double, P_d]
    L.orc_topology.restype = C.c_int
    L.orc_topology.argtypes = [C.POINTER(OrcLigand), P_u8, P_i32]
    L.orc_quat_matrix.restype = None
    L.orc_quat_matrix.argtypes = [P_d, P_d]
    L.orc_pose.restype = None
    L.orc_pose.argtypes = [C.POINTER(OrcLigand), P_u8, P_f, P_d, C.c_int, P_d]
    L.orc_intra.restype = C.c_double
    L.orc_intra.argtypes = [C.POINTER(OrcLigand), C.POINTER(OrcParams), P_i32, C.c_int, P_d, P_d]
    L.orc_inter_pairwise.restype = C.c_double
    L.orc_inter_pairwise.argtypes = [C.POINTER(OrcLigand), C.POINTER(OrcParams),
                                     C.POINTER(OrcPocket), P_d]
    L.orc_grid_geometry.restype = None
    L.orc_grid_geometry.argtypes = [C.POINTER(OrcPocket), C.c_int32, C.POINTER(OrcGrid)]
    L.orc_grid_build.restype = None
    L.orc_grid_build.argtypes = [C.POINTER(OrcPocket), C.POINTER(OrcParams), C.POINTER(OrcGrid),
                                 C.c_int]
    L.orc_trilinear.restype = C.c_int
    L.orc_trilinear.argtypes = [C.POINTER(OrcGrid), P_d, C.c_double, C.c_double, C.c_double, P_d]
    L.orc_inter_grid.restype = C.c_double
    L.orc_inter_grid.argtypes = [C.POINTER(OrcLigand), C.POINTER(OrcGrid), P_d, P_d]
    L.orc_score_poses.restype = C.c_int
    L.orc_score_poses.argtypes = [C.POINTER(OrcLigand), C.POINTER(OrcParams), C.POINTER(OrcGrid),
                                  P_d, P_f, C.c_int, C.c_int64, P_d, P_d, P_d, P_d, P_d]
    L.orc_philox4x64.restype = None
    L.orc_philox4x64.argtypes = [P_u64, P_u64, P_u64]
    L.orc_rng_words.restype = None
    L.orc_rng_words.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                C.POINTER(C.c_uint32)]
    L.orc_normal.restype = C.c_float
    L.orc_normal.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
    L.orc_ga_init.restype = None
    L.orc_ga_init.argtypes = [C.c_int, C.c_int, C.c_float, C.c_uint64, C.c_uint64, P_f]
    L.orc_ga_step.restype = None
    L.orc_ga_step.argtypes = [C.c_int, C.c_int, C.c_float, C.c_float, C.c_uint64, C.c_uint64,
                              C.c_uint32, P_f, P_f, P_f]
    L.orc_ga_children.restype = None
    L.orc_ga_children.argtypes = [C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_uint64,
                                  C.c_uint64, C.c_uint32, P_f, P_f, P_f]
    L.orc_ls_normal.restype = C.c_float
    L.orc_ls_normal.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int]
    L.orc_ls_selected.restype = C.c_int
    L.orc_ls_selected.argtypes = [C.c_float, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32]
    L.orc_solis_wets.restype = C.c_int
    L.orc_solis_wets.argtypes = [C.c_int, C.POINTER(OrcLsParams), C.c_uint64, C.c_uint64,
                                 C.c_uint32, C.c_uint32, P_f, P_f, LS_OBJECTIVE, C.c_void_p,
                                 P_i32]
    L.orc_dock_batch.restype = None
    L.orc_dock_batch.argtypes = [C.POINTER(OrcBatch), C.POINTER(OrcParams), C.POINTER(OrcPocket),
                                 C.POINTER(OrcGrid), C.POINTER(OrcSearch), C.c_int, P_f, P_f, P_d,
                                 P_i32]
    if hasattr(L, "orc_features"):
        _declare_surrogate(L)


def _declare_surrogate(L):
    L.orc_features.restype = None
    L.orc_features.argtypes = [C.POINTER(OrcLigand), P_d, P_d, P_f, C.c_double, P_d]
    L.orc_mlp_forward.restype = None
    L.orc_mlp_forward.argtypes = [P_d, C.c_int, P_d, P_d]
    L.orc_mlp_backward.restype = C.c_double
    L.orc_mlp_backward.argtypes = [P_d, C.c_int, P_d, P_d, P_d]
    L.orc_mlp_n_params.restype = C.c_int
    L.orc_mlp_n_params.argtypes = []
    L.orc_adam_step.restype = None
    L.orc_adam_step.argtypes = [P_d, P_d, P_d, P_d, C.c_int64, C.c_double, C.c_double, C.c_double,
                                C.c_double, C.c_int]
    L.orc_train_order.restype = None
    L.orc_train_order.argtypes = [C.c_uint64, C.c_int64, P_i64]


def _p(a, t):
    return a.ctypes.data_as(t)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------------------
# Wrapped objects (keep numpy buffers alive beside the struct)
# ---------------------------------------------------------------------------
class Params:
    def __init__(self, table: dict):
        self.a = {k: _c(table[k], np.int32 if k == "hb_role" else np.float32) for k in
                  ("Rii", "eps", "vol", "solpar", "hb_R", "hb_eps", "hb_role")}
        self.n_types = int(self.a["Rii"].shape[0])
        self.s = OrcParams(self.n_types, *[_p(self.a[k], P_f) for k in
                                           ("Rii", "eps", "vol", "solpar", "hb_R", "hb_eps")],
                           _p(self.a["hb_role"], P_i32))


class Ligand:
    def __init__(self, x, y, z, q, type, parent, tors_b, **_):
        self.a = dict(x=_c(x, np.float32), y=_c(y, np.float32), z=_c(z, np.float32),
                      q=_c(q, np.float32), type=_c(type, np.uint8), parent=_c(parent, np.int16),
                      tors_b=_c(tors_b, np.int16))
        self.n = int(self.a["x"].shape[0])
        self.k = int(self.a["tors_b"].shape[0])
        a = self.a
        self.s = OrcLigand(self.n, _p(a["x"], P_f), _p(a["y"], P_f), _p(a["z"], P_f),
                           _p(a["q"], P_f), _p(a["type"], P_u8), _p(a["parent"], P_i16), self.k,
                           _p(a["tors_b"], P_i16))

    @property
    def n_genes(self):
        return 7 + self.k


class PocketS:
    def __init__(self, x, y, z, q, type, center, radius, spacing=0.375):
        self.a = dict(x=_c(x, np.float32), y=_c(y, np.float32), z=_c(z, np.float32),
                      q=_c(q, np.float32), type=_c(type, np.uint8))
        a = self.a
        self.center = np.asarray(center, np.float64)
        self.radius = float(radius)
        self.spacing = float(spacing)
        self.s = OrcPocket(int(a["x"].shape[0]), _p(a["x"], P_f), _p(a["y"], P_f), _p(a["z"], P_f),
                           _p(a["q"], P_f), _p(a["type"], P_u8),
                           (C.c_double * 3)(*self.center), self.radius, self.spacing)


def pocket_from(pk) -> PocketS:
    return PocketS(pk.x, pk.y, pk.z, pk.q, pk.type, pk.center, pk.radius, pk.spacing)


@dataclass
class Grid:
    s: OrcGrid
    maps: np.ndarray       # [T+2, nz, ny, nx] float64

    @property
    def n(self):
        return (self.s.nx, self.s.ny, self.s.nz)

    @property
    def origin(self):
        return np.array([self.s.ox, self.s.oy, self.s.oz])

    @property
    def h(self):
        return self.s.h


# ---------------------------------------------------------------------------
# Functions
# ---------------------------------------------------------------------------
def dielectric(r: float) -> float:
    return lib().orc_dielectric(r)


def disp_raw(params: Params, ti: int, tj: int, r: float) -> float:
    return lib().orc_disp_raw(C.byref(params.s), ti, tj, r)


def pair_terms(params: Params, ti, tj, qi, qj, r) -> np.ndarray:
    out = np.zeros(4, np.float64)
    lib().orc_pair_terms(C.byref(params.s), int(ti), int(tj), float(qi), float(qj), float(r),
                         _p(out, P_d))
    return out


def topology(lig: Ligand):
    n, k = lig.n, lig.k
    moves = np.zeros(max(k, 1) * n, np.uint8)
    pairs = np.zeros(n * (n - 1) + 2, np.int32)
    np_ = lib().orc_topology(C.byref(lig.s), _p(moves, P_u8), _p(pairs, P_i32))
    if np_ < 0:
        raise ValueError("bad ligand topology")
    return moves[:k * n].reshape(k, n).astype(bool), pairs[:2 * np_].reshape(np_, 2)


def _moves_arg(lig: Ligand):
    n, k = lig.n, lig.k
    moves = np.zeros(max(k, 1) * n, np.uint8)
    pairs = np.zeros(n * (n - 1) + 2, np.int32)
    np_ = lib().orc_topology(C.byref(lig.s), _p(moves, P_u8), _p(pairs, P_i32))
    if np_ < 0:
        raise ValueError("bad ligand topology")
    return moves, pairs, np_


def quat_matrix(q) -> np.ndarray:
    q = _c(q, np.float64)
    R = np.zeros(9, np.float64)
    lib().orc_quat_matrix(_p(q, P_d), _p(R, P_d))
    return R.reshape(3, 3)


def pose(lig: Ligand, geno, center, order: int = 0) -> np.ndarray:
    moves, _, _ = _moves_arg(lig)
    g = _c(geno, np.float32)
    c = _c(center, np.float64)
    xyz = np.zeros(3 * lig.n, np.float64)
    lib().orc_pose(C.byref(lig.s), _p(moves, P_u8), _p(g, P_f), _p(c, P_d), order, _p(xyz, P_d))
    return xyz.reshape(lig.n, 3)


def intra(lig: Ligand, params: Params, xyz):
    _, pairs, np_ = _moves_arg(lig)
    x = _c(xyz, np.float64)
    m = C.c_double()
    e = lib().orc_intra(C.byref(lig.s), C.byref(params.s), _p(pairs, P_i32), np_, _p(x, P_d),
                        C.byref(m))
    return e, m.value


def inter_pairwise(lig: Ligand, params: Params, pocket: PocketS, xyz) -> float:
    x = _c(xyz, np.float64)
    return lib().orc_inter_pairwise(C.byref(lig.s), C.byref(params.s), C.byref(pocket.s), _p(x, P_d))


def grid_geometry(pocket: PocketS, n_types: int) -> OrcGrid:
    g = OrcGrid()
    lib().orc_grid_geometry(C.byref(pocket.s), n_types, C.byref(g))
    return g


def grid_build(pocket: PocketS, params: Params, n_threads: int = 0) -> Grid:
    g = grid_geometry(pocket, params.n_types)
    maps = np.zeros((params.n_types + 2, g.nz, g.ny, g.nx), np.float64)
    g.maps = _p(maps, P_d)
    lib().orc_grid_build(C.byref(pocket.s), C.byref(params.s), C.byref(g),
                         n_threads or (os.cpu_count() or 1))
    return Grid(g, maps)


def grid_with_maps(geom: OrcGrid, maps: np.ndarray) -> Grid:
    """A Grid with the given geometry and caller-provided maps."""
    maps = _c(maps, np.float64)
    g = OrcGrid(geom.nx, geom.ny, geom.nz, geom.n_types, geom.ox, geom.oy, geom.oz, geom.h,
                _p(maps, P_d))
    return Grid(g, maps)


def trilinear(grid: Grid, map_index: int, x, y, z):
    vol = grid.s.nx * grid.s.ny * grid.s.nz
    base = C.cast(grid.s.maps, C.c_void_p).value + 8 * vol * map_index
    v = C.c_double()
    out = lib().orc_trilinear(C.byref(grid.s), C.cast(base, P_d), float(x), float(y), float(z),
                              C.byref(v))
    return None if out else v.value


def inter_grid(lig: Ligand, grid: Grid, xyz):
    x = _c(xyz, np.float64)
    m = C.c_double()
    e = lib().orc_inter_grid(C.byref(lig.s), C.byref(grid.s), _p(x, P_d), C.byref(m))
    return e, m.value


def score_poses(lig: Ligand, params: Params, grid: Grid, center, genos, want_xyz=False):
    g = _c(genos, np.float32).reshape(-1, lig.n_genes)
    n = g.shape[0]
    c = _c(center, np.float64)
    out = {k: np.zeros(n, np.float64) for k in ("score", "inter", "intra", "margin")}
    xyz = np.zeros((n, lig.n, 3), np.float64) if want_xyz else None
    np_ = lib().orc_score_poses(C.byref(lig.s), C.byref(params.s), C.byref(grid.s), _p(c, P_d),
                                _p(g, P_f), lig.n_genes, n, _p(out["score"], P_d),
                                _p(out["inter"], P_d), _p(out["intra"], P_d),
                                _p(out["margin"], P_d), _p(xyz, P_d) if want_xyz else None)
    if np_ < 0:
        raise ValueError("bad ligand topology")
    out["n_pairs"] = np_
    if want_xyz:
        out["xyz"] = xyz
    return out


def philox4x64(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint64)
    k = _c(key, np.uint64)
    o = np.zeros(4, np.uint64)
    lib().orc_philox4x64(_p(c, P_u64), _p(k, P_u64), _p(o, P_u64))
    return o


def rng_words(seed, lig, gen, ind, slot) -> np.ndarray:
    w = (C.c_uint32 * 8)()
    lib().orc_rng_words(seed, lig, gen, ind, slot, w)
    return np.array(list(w), np.uint32)


def normal(seed, lig, gen, ind, slot) -> float:
    return lib().orc_normal(seed, lig, gen, ind, slot)


def ga_init(k: int, pop: int, radius: float, seed: int, lig_id: int) -> np.ndarray:
    g = np.zeros(pop * (7 + k), np.float32)
    lib().orc_ga_init(k, pop, radius, seed, lig_id, _p(g, P_f))
    return g.reshape(pop, 7 + k)


def ga_step(k: int, pop: int, p_cross: float, p_mut: float, seed: int, lig_id: int, gen: int,
            prev, scores) -> np.ndarray:
    prev = _c(prev, np.float32)
    sc = _c(scores, np.float32)
    nxt = np.zeros(pop * (7 + k), np.float32)
    lib().orc_ga_step(k, pop, p_cross, p_mut, seed, lig_id, gen, _p(prev, P_f), _p(sc, P_f),
                      _p(nxt, P_f))
    return nxt.reshape(pop, 7 + k)


def ga_children(k: int, pop: int, n: int, p_cross: float, p_mut: float, seed: int, lig_id: int,
                gen: int, prev, scores) -> np.ndarray:
    prev = _c(prev, np.float32)
    sc = _c(scores, np.float32)
    out = np.zeros(n * (7 + k), np.float32)
    lib().orc_ga_children(k, pop, n, p_cross, p_mut, seed, lig_id, gen, _p(prev, P_f), _p(sc, P_f),
                          _p(out, P_f))
    return out.reshape(n, 7 + k)


class LsParams:
    """Solis-Wets settings; the defaults are AutoDock's published ones (Morris et
    al. 1998): 6% of the individuals per generation, at most 300 iterations,
    rho doubled after 4 successes and halved after 4 failures in a row, from
    1.0 down to 0.01."""

    def __init__(self, rate=0.06, max_its=300, max_succ=4, max_fail=4, rho=1.0, rho_lb=0.01):
        self.s = OrcLsParams(rate, max_its, max_succ, max_fail, rho, rho_lb)


def ls_selected(rate: float, seed: int, lig_id: int, gen: int, ind: int) -> bool:
    """Whether individual `ind` of generation `gen` is refined (Solis-Wets)."""
    return bool(lib().orc_ls_selected(rate, seed, lig_id, gen, ind))


def ls_normal(seed: int, lig_id: int, gen: int, ind: int, t: int, e: int) -> float:
    """The local search's N(0, 1) draw for gene e at iteration t."""
    return lib().orc_ls_normal(seed, lig_id, gen, ind, t, e)


def solis_wets(k: int, ls: LsParams, seed: int, lig_id: int, gen: int, ind: int, x0, f0,
               objective):
    """Solis-Wets local search of one individual (oracle.c states the steps).
    objective(genotype float32[7 + k], iteration, which) -> score, which = 0
    for the probe x + xi and 1 for x - xi. Returns (x, f, iterations, evals)."""
    x = np.array(x0, np.float32).reshape(7 + k).copy()
    f = np.array([f0], np.float32)
    err = []

    def cb(g, it, which, _ctx):
        try:
            return float(objective(np.ctypeslib.as_array(g, (7 + k,)).copy(), it, which))
        except Exception as e:  # noqa: BLE001 - reported after the C call returns
            err.append(e)
            return float("nan")
    fn = LS_OBJECTIVE(cb)
    its = C.c_int32(0)
    ev = lib().orc_solis_wets(k, C.byref(ls.s), seed, lig_id, gen, ind, _p(x, P_f), _p(f, P_f),
                              fn, None, C.byref(its))
    if err:
        raise err[0]
    return x, float(f[0]), int(its.value), int(ev)


def _order_key(scores):
    """Sort key of FP32 scores: NaN counts as +inf (the GA's comparison)."""
    s = np.asarray(scores, np.float32).astype(np.float64)
    return np.where(np.isnan(s), np.inf, s)


def topk(pred, keep: int) -> np.ndarray:
    """Indices of the `keep` lowest predictions, ties by index."""
    idx = np.arange(len(pred))
    return np.lexsort((idx, _order_key(pred)))[:keep]


def merge(pop_scores, kept_scores, pop: int):
    """mu + lambda: (origin, index) of the best `pop` of population (origin 0)
    and kept candidates (origin 1) by score, ties by origin then index."""
    s = np.concatenate([_order_key(pop_scores), _order_key(kept_scores)])
    origin = np.concatenate([np.zeros(len(pop_scores), int), np.ones(len(kept_scores), int)])
    index = np.concatenate([np.arange(len(pop_scores)), np.arange(len(kept_scores))])
    order = np.lexsort((index, origin, s))[:pop]
    return origin[order], index[order]


def dock_batch(ligs, params: Params, pocket: PocketS, grid: Grid, pop: int, generations: int,
               p_cross: float = 0.8, p_mut: float = 0.02, seed: int = 0, n_threads: int = 0,
               ls: LsParams | None = None):
    """Free-run search over a CSR ligand set (synth.LigandSet fields); with
    `ls`, the Lamarckian variant (Solis-Wets on the selected individuals of
    every generation, the oracle's own FP32-rounded scores as objective)."""
    a = dict(atom_off=_c(ligs.atom_off, np.int32), tors_off=_c(ligs.tors_off, np.int32),
             x=_c(ligs.x, np.float32), y=_c(ligs.y, np.float32), z=_c(ligs.z, np.float32),
             q=_c(ligs.q, np.float32), type=_c(ligs.type, np.uint8),
             parent=_c(ligs.parent, np.int16), tors_b=_c(ligs.tors_b, np.int16),
             ligand_id=_c(ligs.ligand_id, np.uint64))
    nl = int(a["atom_off"].shape[0] - 1)
    b = OrcBatch(nl, _p(a["atom_off"], P_i32), _p(a["tors_off"], P_i32), _p(a["x"], P_f),
                 _p(a["y"], P_f), _p(a["z"], P_f), _p(a["q"], P_f), _p(a["type"], P_u8),
                 _p(a["parent"], P_i16), _p(a["tors_b"], P_i16), _p(a["ligand_id"], P_u64))
    s = OrcSearch(pop, generations, p_cross, p_mut, seed,
                  ls.s if ls is not None else OrcLsParams(0.0, 0, 1, 1, 1.0, 0.0))
    geno = np.zeros((nl, pop, 23), np.float32)
    score = np.zeros((nl, pop), np.float32)
    best64 = np.zeros((nl, 8), np.float64)
    best_idx = np.zeros((nl, 8), np.int32)
    nt = n_threads or (os.cpu_count() or 1)
    lib().orc_dock_batch(C.byref(b), C.byref(params.s), C.byref(pocket.s), C.byref(grid.s),
                         C.byref(s), nt, _p(geno, P_f), _p(score, P_f), _p(best64, P_d),
                         _p(best_idx, P_i32))
    return dict(geno=geno, score=score, best64=best64, best_idx=best_idx, threads=nt)


# ---------------------------------------------------------------------------
# Surrogate (features, MLP): oracle/surrogate.c
# ---------------------------------------------------------------------------
N_FEATURES, N_HIDDEN = 128, 256


def to_bf16(a) -> np.ndarray:
    """Round to bfloat16 (round to nearest even, via float32) and return the
    values as float64: float64 -> float32 (RN) -> bfloat16 (RNE)."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def features(lig: Ligand, xyz, center, geno, radius) -> np.ndarray:
    """FP64 features of one posed ligand (before any rounding)."""
    x = _c(xyz, np.float64)
    c = _c(center, np.float64)
    g = _c(geno, np.float32)
    f = np.zeros(N_FEATURES, np.float64)
    lib().orc_features(C.byref(lig.s), _p(x, P_d), _p(c, P_d), _p(g, P_f), float(radius), _p(f, P_d))
    return f


def mlp_n_params() -> int:
    return lib().orc_mlp_n_params()


def mlp_unpack(p):
    """Split packed parameters into (W1, b1, W2, b2, W3, b3, W4, b4)."""
    F, H = N_FEATURES, N_HIDDEN
    sizes = [(F, H), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)]
    out, o = [], 0
    for sh in sizes:
        n = int(np.prod(sh))
        out.append(np.asarray(p[o:o + n]).reshape(sh))
        o += n
    return out


def mlp_forward(params, X) -> np.ndarray:
    p = _c(params, np.float64)
    X = _c(X, np.float64).reshape(-1, N_FEATURES)
    Y = np.zeros(X.shape[0], np.float64)
    lib().orc_mlp_forward(_p(p, P_d), X.shape[0], _p(X, P_d), _p(Y, P_d))
    return Y


def mlp_backward(params, X, T):
    p = _c(params, np.float64)
    X = _c(X, np.float64).reshape(-1, N_FEATURES)
    T = _c(T, np.float64)
    g = np.zeros_like(p)
    loss = lib().orc_mlp_backward(_p(p, P_d), X.shape[0], _p(X, P_d), _p(T, P_d), _p(g, P_d))
    return loss, g


def adam_step(p, m, v, g, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One FP64 Adam step in place on float64 arrays p, m, v (step t >= 1)."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _c(g, np.float64)
    lib().orc_adam_step(_p(p, P_d), _p(m, P_d), _p(v, P_d), _p(g, P_d), p.size, lr, b1, b2, eps, t)


def train_order(seed: int, n: int) -> np.ndarray:
    """Row visited at each position of a training run (a permutation of n)."""
    out = np.zeros(n, np.int64)
    lib().orc_train_order(C.c_uint64(seed), n, _p(out, P_i64))
    return out


def standardize_targets(scores, clip: float):
    """(mean, std) of min(score, clip) over the training set, in FP64."""
    t = np.minimum(np.asarray(scores, np.float64), clip)
    mean = t.mean()
    return mean, float(np.sqrt(max((t * t).mean() - mean * mean, 1e-12)))


# ---------------------------------------------------------------------------
# FP32 auto-vectorised CPU baseline (simd_fp32.c): a second CPU reference
# point for the benchmark, not part of the oracle's parity role
# ---------------------------------------------------------------------------
def cpu32_score_poses(lig: Ligand, params: Params, grid: Grid, center, genos) -> np.ndarray:
    g = _c(genos, np.float32).reshape(-1, lig.n_genes)
    out = np.zeros(g.shape[0], np.float32)
    c = _c(center, np.float64)
    if lib32().cpu32_score_poses(C.byref(lig.s), C.byref(params.s), C.byref(grid.s), _p(c, P_d),
                                 _p(g, P_f), lig.n_genes, g.shape[0], _p(out, P_f)) < 0:
        raise ValueError("bad ligand topology")
    return out


def cpu32_dock_batch(ligs, params: Params, pocket: PocketS, grid: Grid, pop: int, generations: int,
                     p_cross: float = 0.8, p_mut: float = 0.02, seed: int = 0, n_threads: int = 0,
                     trace: bool = False):
    """The plain GA search with FP32 auto-vectorised scoring; with trace, the
    genotypes and scores of every generation of ligand 0."""
    a = dict(atom_off=_c(ligs.atom_off, np.int32), tors_off=_c(ligs.tors_off, np.int32),
             x=_c(ligs.x, np.float32), y=_c(ligs.y, np.float32), z=_c(ligs.z, np.float32),
             q=_c(ligs.q, np.float32), type=_c(ligs.type, np.uint8),
             parent=_c(ligs.parent, np.int16), tors_b=_c(ligs.tors_b, np.int16),
             ligand_id=_c(ligs.ligand_id, np.uint64))
    nl = int(a["atom_off"].shape[0] - 1)
    b = OrcBatch(nl, _p(a["atom_off"], P_i32), _p(a["tors_off"], P_i32), _p(a["x"], P_f),
                 _p(a["y"], P_f), _p(a["z"], P_f), _p(a["q"], P_f), _p(a["type"], P_u8),
                 _p(a["parent"], P_i16), _p(a["tors_b"], P_i16), _p(a["ligand_id"], P_u64))
    score = np.zeros((nl, pop), np.float32)
    best = np.zeros(nl, np.int32)
    G0 = 7 + int(a["tors_off"][1] - a["tors_off"][0]) if nl else 7
    tg = np.zeros((generations, pop, G0), np.float32) if trace else None
    ts = np.zeros((generations, pop), np.float32) if trace else None
    nt = n_threads or (os.cpu_count() or 1)
    lib32().cpu32_dock_batch(C.byref(b), C.byref(params.s), C.byref(pocket.s), C.byref(grid.s),
                             pop, generations, p_cross, p_mut, seed, nt, _p(score, P_f),
                             _p(best, P_i32), _p(tg, P_f) if trace else None,
                             _p(ts, P_f) if trace else None)
    return dict(score=score, best=best, trace_geno=tg, trace_score=ts, threads=nt)
