"""Python binding of libdock.so (include/dock.h): argument marshalling only.

Every step of the docking path runs in the library's CUDA kernels; this
module converts numpy arrays and torch tensors to the C structs and pointers
the ABI takes. It raises if the compiled library is missing: there is no
Python or CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# DOCK_CHECKED=1 in the environment loads the bounds-checked build instead
# (libdock_checked.so, made by build.build(checked=True)).
LIB_PATH = os.path.join(_PKG, "libdock_checked.so" if os.environ.get("DOCK_CHECKED") == "1"
                        else "libdock.so")

DOCK_OK, DOCK_EINVAL, DOCK_ENOMEM, DOCK_ECUDA, DOCK_ETIMEOUT, DOCK_EDEVICE, DOCK_ENOTIMPL = \
    0, -1, -2, -3, -4, -5, -6
DOCK_MAX_ATOMS, DOCK_MAX_TORSIONS, DOCK_MAX_GENES, DOCK_MAX_TYPES, DOCK_N_BEST = 128, 16, 23, 16, 8

P_f = C.POINTER(C.c_float)
P_u8 = C.POINTER(C.c_uint8)
P_i16 = C.POINTER(C.c_int16)
P_i32 = C.POINTER(C.c_int32)
P_u64 = C.POINTER(C.c_uint64)


class DockError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("dock status %d: %s" % (status, msg))
        self.status = status


class dock_type_params(C.Structure):
    _fields_ = [("Rii", C.c_float), ("eps", C.c_float), ("vol", C.c_float), ("solpar", C.c_float),
                ("hb_R", C.c_float), ("hb_eps", C.c_float), ("hb_role", C.c_int32)]


class dock_pocket_desc(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("x", P_f), ("y", P_f), ("z", P_f), ("q", P_f),
                ("type", P_u8), ("center", C.c_float * 3), ("radius", C.c_float),
                ("spacing", C.c_float), ("n_types", C.c_int32),
                ("params", C.POINTER(dock_type_params))]


class dock_ligand_batch(C.Structure):
    _fields_ = [("n_ligands", C.c_int32), ("atom_off", P_i32), ("x", P_f), ("y", P_f), ("z", P_f),
                ("q", P_f), ("type", P_u8), ("parent", P_i16), ("tors_off", P_i32),
                ("tors_b", P_i16), ("ligand_id", P_u64)]


class dock_ls_params(C.Structure):
    _fields_ = [("rate", C.c_float), ("max_its", C.c_int32), ("max_succ", C.c_int32),
                ("max_fail", C.c_int32), ("rho", C.c_float), ("rho_lb", C.c_float)]


def ls_params(rate=0.06, max_its=300, max_succ=4, max_fail=4, rho=1.0, rho_lb=0.01):
    """Solis-Wets settings (AutoDock's published defaults)."""
    return dock_ls_params(rate, max_its, max_succ, max_fail, rho, rho_lb)


NO_LS = (0.0, 300, 4, 4, 1.0, 0.01)


class dock_search_params(C.Structure):
    _fields_ = [("pop", C.c_int32), ("generations", C.c_int32), ("p_cross", C.c_float),
                ("p_mut", C.c_float), ("seed", C.c_uint64), ("lanes_per_pose", C.c_int32),
                ("use_graph", C.c_int32), ("timeout_ns", C.c_uint64),
                ("trace_genotypes", C.c_void_p), ("trace_scores", C.c_void_p),
                ("mode", C.c_int32), ("candidates", C.c_int32), ("keep", C.c_int32),
                ("surrogate", C.c_void_p), ("ls", dock_ls_params), ("trace_ls", C.c_void_p),
                ("inter", C.c_int32), ("resume_genotypes", C.c_void_p),
                ("resume_scores", C.c_void_p), ("resume_from", C.c_int32)]


DOCK_INTER_GRID, DOCK_INTER_PAIRWISE = 0, 1


DOCK_TUNE_MAX = 16


class dock_tune_table(C.Structure):
    _fields_ = [("n", C.c_int32), ("threads", C.c_int32 * DOCK_TUNE_MAX),
                ("atoms_per_lane", C.c_int32 * DOCK_TUNE_MAX),
                ("ms_per_generation", C.c_float * DOCK_TUNE_MAX), ("best", C.c_int32)]


class dock_train_params(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float),
                ("score_clip", C.c_float), ("seed", C.c_uint64)]


DOCK_MODE_PLAIN, DOCK_MODE_SURROGATE = 0, 1
DOCK_N_FEATURES, DOCK_MLP_N_PARAMS = 128, 164865


class dock_result(C.Structure):
    _fields_ = [("ligand_id", C.c_uint64), ("n_genes", C.c_int32), ("status", C.c_int32),
                ("best_fp32", C.c_float * DOCK_N_BEST), ("best_fp64", C.c_double * DOCK_N_BEST),
                ("best_index", C.c_int32 * DOCK_N_BEST),
                ("genotype", (C.c_float * DOCK_MAX_GENES) * DOCK_N_BEST),
                ("exact_evals", C.c_uint64), ("surrogate_evals", C.c_uint64)]


RESULT_DTYPE = np.dtype([("ligand_id", np.uint64), ("n_genes", np.int32), ("status", np.int32),
                         ("best_fp32", np.float32, DOCK_N_BEST),
                         ("best_fp64", np.float64, DOCK_N_BEST),
                         ("best_index", np.int32, DOCK_N_BEST),
                         ("genotype", np.float32, (DOCK_N_BEST, DOCK_MAX_GENES)),
                         ("exact_evals", np.uint64), ("surrogate_evals", np.uint64)], align=True)

_lib = None


def lib():
    """Load libdock.so (built by paper_2509_12232_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built: run paper_2509_12232_gb300.build.build() "
                               "(nvcc, sm_103a); there is no CPU fallback"
                               % os.path.basename(LIB_PATH))
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.dock_last_error.restype = C.c_char_p
        L.dock_version.restype = C.c_char_p
        L.dock_create_pocket.argtypes = [C.POINTER(dock_pocket_desc), vp, C.POINTER(vp)]
        L.dock_pocket_destroy.argtypes = [vp]
        L.dock_pocket_destroy.restype = None
        L.dock_pocket_grid.argtypes = [vp, P_i32, P_f, C.POINTER(vp)]
        L.dock_load_ligands.argtypes = [vp, C.POINTER(dock_ligand_batch), vp, C.POINTER(vp)]
        L.dock_ligands_destroy.argtypes = [vp]
        L.dock_ligands_destroy.restype = None
        L.dock_batch.argtypes = [vp, vp, C.POINTER(dock_search_params), vp, C.POINTER(vp)]
        L.dock_results.argtypes = [vp, vp, C.c_int32, C.c_uint64]
        L.dock_job_population.argtypes = [vp, C.POINTER(vp), C.POINTER(vp)]
        L.dock_job_kernel_time.argtypes = [vp, C.POINTER(C.c_double), P_i32]
        L.dock_job_destroy.argtypes = [vp]
        L.dock_job_destroy.restype = None
        L.dock_score.argtypes = [vp, vp, vp, vp, C.c_int64, vp, vp, vp, C.c_int32, vp]
        L.dock_score_pairwise.argtypes = [vp, vp, vp, vp, C.c_int64, vp, vp]
        L.dock_local_search.argtypes = [vp, vp, C.POINTER(dock_ls_params), C.c_uint64, C.c_uint32,
                                        vp, C.c_int64, vp, vp, vp, vp, vp]
        P_i64 = C.POINTER(C.c_int64)
        L.dock_ligands_info.argtypes = [vp, P_i32, P_i64, P_i64, P_i64, P_i64, P_i64]
        L.dock_batch_noalloc.argtypes = [vp, vp, C.POINTER(dock_search_params), vp, vp]
        L.dock_features.argtypes = [vp, vp, vp, vp, C.c_int64, vp, vp, vp]
        L.dock_autotune.argtypes = [vp, vp, C.POINTER(dock_search_params), vp,
                                    C.POINTER(dock_tune_table)]
        L.dock_features_population.argtypes = [vp, vp, C.c_int32, vp, vp, vp, vp]
        L.dock_surrogate_create.argtypes = [C.c_uint64, vp, C.POINTER(vp)]
        L.dock_surrogate_destroy.argtypes = [vp]
        L.dock_surrogate_destroy.restype = None
        L.dock_surrogate_set_params.argtypes = [vp, vp, C.c_float, C.c_float, C.c_float, vp]
        L.dock_surrogate_get_params.argtypes = [vp, vp, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                                C.POINTER(C.c_float)]
        L.dock_surrogate_predict.argtypes = [vp, vp, C.c_int64, vp, vp]
        L.dock_surrogate_gradients.argtypes = [vp, vp, vp, C.c_int32, vp, C.POINTER(C.c_float), vp]
        L.dock_surrogate_train.argtypes = [vp, vp, vp, C.c_int64, C.POINTER(dock_train_params), vp,
                                           vp]
        L.dock_measure_peaks.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        for name in ("dock_create_pocket", "dock_pocket_grid", "dock_load_ligands", "dock_batch",
                     "dock_results", "dock_job_population", "dock_job_kernel_time", "dock_score",
                     "dock_score_pairwise",
                     "dock_ligands_info", "dock_batch_noalloc", "dock_features",
                     "dock_features_population", "dock_surrogate_create",
                     "dock_surrogate_set_params", "dock_surrogate_get_params",
                     "dock_surrogate_predict", "dock_surrogate_gradients",
                     "dock_surrogate_train", "dock_autotune", "dock_measure_peaks"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def check(status: int):
    if status != DOCK_OK:
        raise DockError(status, lib().dock_last_error().decode())


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _p(a, t):
    return a.ctypes.data_as(t)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _dptr(t):
    """Device pointer of a torch tensor (or an int), None for None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(int(t))


class Pocket:
    """Owns a dock_pocket handle."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def grid(self):
        n = C.c_int32()
        o = (C.c_float * 3)()
        maps = C.c_void_p()
        check(lib().dock_pocket_grid(self.handle, C.byref(n), o, C.byref(maps)))
        return n.value, np.array(list(o), np.float32), maps.value

    def close(self):
        if self.handle:
            lib().dock_pocket_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ligands:
    def __init__(self, handle, n_ligands, n_tors):
        self.handle = handle
        self.n_ligands = n_ligands
        self.n_tors = n_tors

    def geno_offsets(self, pop: int) -> np.ndarray:
        g = (7 + self.n_tors.astype(np.int64)) * pop
        return np.concatenate([[0], np.cumsum(g)]).astype(np.int64)

    def close(self):
        if self.handle:
            lib().dock_ligands_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Job:
    def __init__(self, handle, n_ligands, keep=()):
        self.handle = handle
        self.n_ligands = n_ligands
        self._keep = keep          # the pocket and ligands must outlive the job

    def close(self):
        if self.handle:
            lib().dock_job_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def type_params_array(table: dict):
    n = len(table["Rii"])
    arr = (dock_type_params * n)()
    for t in range(n):
        arr[t] = dock_type_params(float(table["Rii"][t]), float(table["eps"][t]),
                                  float(table["vol"][t]), float(table["solpar"][t]),
                                  float(table["hb_R"][t]), float(table["hb_eps"][t]),
                                  int(table["hb_role"][t]))
    return arr


def dock_create_pocket(x, y, z, q, type, center, radius, spacing, params_table, stream=None) -> Pocket:
    keep = dict(x=_c(x, np.float32), y=_c(y, np.float32), z=_c(z, np.float32), q=_c(q, np.float32),
                type=_c(type, np.uint8))
    params = type_params_array(params_table)
    d = dock_pocket_desc(int(keep["x"].shape[0]), _p(keep["x"], P_f), _p(keep["y"], P_f),
                         _p(keep["z"], P_f), _p(keep["q"], P_f), _p(keep["type"], P_u8),
                         (C.c_float * 3)(*[float(c) for c in center]), float(radius), float(spacing),
                         len(params), params)
    h = C.c_void_p()
    check(lib().dock_create_pocket(C.byref(d), _stream(stream), C.byref(h)))
    return Pocket(h, keep)


def dock_load_ligands(pocket: Pocket, atom_off, x, y, z, q, type, parent, tors_off, tors_b, ligand_id,
                      stream=None) -> Ligands:
    a = dict(atom_off=_c(atom_off, np.int32), x=_c(x, np.float32), y=_c(y, np.float32),
             z=_c(z, np.float32), q=_c(q, np.float32), type=_c(type, np.uint8),
             parent=_c(parent, np.int16), tors_off=_c(tors_off, np.int32),
             tors_b=_c(tors_b, np.int16), ligand_id=_c(ligand_id, np.uint64))
    nl = int(a["atom_off"].shape[0] - 1)
    b = dock_ligand_batch(nl, _p(a["atom_off"], P_i32), _p(a["x"], P_f), _p(a["y"], P_f),
                          _p(a["z"], P_f), _p(a["q"], P_f), _p(a["type"], P_u8),
                          _p(a["parent"], P_i16), _p(a["tors_off"], P_i32), _p(a["tors_b"], P_i16),
                          _p(a["ligand_id"], P_u64))
    h = C.c_void_p()
    check(lib().dock_load_ligands(pocket.handle, C.byref(b), _stream(stream), C.byref(h)))
    return Ligands(h, nl, np.diff(a["tors_off"]).astype(np.int64))


def dock_ligands_info(ligands: Ligands) -> dict:
    nl = C.c_int32()
    v = [C.c_int64() for _ in range(5)]
    check(lib().dock_ligands_info(ligands.handle, C.byref(nl), *[C.byref(x) for x in v]))
    return dict(n_ligands=nl.value, n_atoms=v[0].value, n_pairs=v[1].value, n_torsions=v[2].value,
                n_moved=v[3].value, h2d_bytes=v[4].value)


def dock_batch(pocket: Pocket, ligands: Ligands, pop: int, generations: int, p_cross=0.8,
               p_mut=0.02, seed=0, lanes_per_pose=0, use_graph=1, timeout_ns=0,
               trace_genotypes=None, trace_scores=None, stream=None, surrogate=None,
               candidates=0, keep=0, ls=None, trace_ls=None, inter=0, resume=None) -> Job:
    """Plain search, or the surrogate pre-screened search when `surrogate` is
    given (`candidates` children per ligand and generation, `keep` of them
    scored exactly). `ls` (a dock_ls_params, e.g. ls_params()) with a rate
    > 0 makes the plain search Lamarckian (Solis-Wets refinement). inter =
    DOCK_INTER_PAIRWISE scores with the pairwise inter-energy (no maps).
    resume = (genotypes, scores, generation): continue a plain search from a
    saved generation (device tensors in the trace layout of one generation)."""
    mode = DOCK_MODE_SURROGATE if surrogate is not None else DOCK_MODE_PLAIN
    rg, rs, rf = (None, None, 0) if resume is None else resume
    sp = dock_search_params(pop, generations, p_cross, p_mut, seed, lanes_per_pose, use_graph,
                            timeout_ns, _dptr(trace_genotypes), _dptr(trace_scores), mode,
                            candidates, keep, surrogate.handle if surrogate is not None else None,
                            ls if ls is not None else dock_ls_params(*NO_LS), _dptr(trace_ls),
                            inter, _dptr(rg), _dptr(rs), rf)
    h = C.c_void_p()
    check(lib().dock_batch(pocket.handle, ligands.handle, C.byref(sp), _stream(stream), C.byref(h)))
    return Job(h, ligands.n_ligands, keep=(pocket, ligands, surrogate))


def dock_batch_noalloc(pocket: Pocket, ligands: Ligands, results, pop: int, generations: int,
                       p_cross=0.8, p_mut=0.02, seed=0, timeout_ns=0, trace_genotypes=None,
                       trace_scores=None, stream=None):
    """The plain search with no device allocation: working buffers live in the
    library's fixed scratch array; `results` is a caller-owned device buffer
    of n_ligands dock_result records (RESULT_DTYPE.itemsize bytes each), a
    CUDA tensor: the kernels write one record per ligand into it and the C
    side cannot see its size, so it is checked here. Asynchronous on stream."""
    need = ligands.n_ligands * RESULT_DTYPE.itemsize
    if not getattr(results, "is_cuda", False):
        raise DockError(DOCK_EINVAL, "dock_batch_noalloc: results must be a CUDA tensor")
    have = int(results.numel()) * int(results.element_size())
    if have < need:
        raise DockError(DOCK_EINVAL, "dock_batch_noalloc: results holds %d bytes, %d ligands need %d"
                        % (have, ligands.n_ligands, need))
    sp = dock_search_params(pop, generations, p_cross, p_mut, seed, 0, 0, timeout_ns,
                            _dptr(trace_genotypes), _dptr(trace_scores), DOCK_MODE_PLAIN, 0, 0,
                            None, dock_ls_params(*NO_LS), None)
    check(lib().dock_batch_noalloc(pocket.handle, ligands.handle, C.byref(sp), _dptr(results),
                                   _stream(stream)))


def dock_results(job: Job, cap: int | None = None, timeout_ns: int = 0) -> np.ndarray:
    cap = job.n_ligands if cap is None else int(cap)
    out = np.zeros(cap, RESULT_DTYPE)
    assert RESULT_DTYPE.itemsize == C.sizeof(dock_result)
    check(lib().dock_results(job.handle, out.ctypes.data_as(C.c_void_p), cap, timeout_ns))
    return out


def dock_job_population(job: Job):
    g, s = C.c_void_p(), C.c_void_p()
    check(lib().dock_job_population(job.handle, C.byref(g), C.byref(s)))
    return g.value, s.value


def dock_job_kernel_time(job: Job):
    ms = C.c_double()
    n = C.c_int32()
    check(lib().dock_job_kernel_time(job.handle, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def dock_score(pocket: Pocket, ligands: Ligands, pose_ligand, genotypes, scores=None, scores64=None,
               coords=None, fp64=False, stream=None):
    """pose_ligand, genotypes ([n, 23] float32), scores / scores64 / coords:
    device tensors (torch) or device pointers; asynchronous on stream."""
    n = int(pose_ligand.shape[0]) if hasattr(pose_ligand, "shape") else int(genotypes.shape[0])
    check(lib().dock_score(pocket.handle, ligands.handle, _dptr(pose_ligand), _dptr(genotypes), n,
                           _dptr(scores), _dptr(scores64), _dptr(coords), 1 if fp64 else 0,
                           _stream(stream)))


def dock_score_pairwise(pocket: Pocket, ligands: Ligands, pose_ligand, genotypes, scores,
                        stream=None):
    """Scores with the pairwise inter-energy (no grid) plus intra-energy of
    genotypes ([n, 23] float32) posed for ligands pose_ligand ([n] int32), all
    device tensors or pointers; asynchronous on stream."""
    n = int(pose_ligand.shape[0]) if hasattr(pose_ligand, "shape") else int(genotypes.shape[0])
    check(lib().dock_score_pairwise(pocket.handle, ligands.handle, _dptr(pose_ligand),
                                    _dptr(genotypes), n, _dptr(scores), _stream(stream)))


def dock_local_search(pocket: Pocket, ligands: Ligands, ls, seed: int, generation: int,
                      pose_ligand, genotypes, scores, trace=None, evals=None, stream=None):
    """Solis-Wets refinement of caller-given poses: genotypes ([n, 23] float32,
    refined in place) of ligands pose_ligand ([n] int32); scores ([n] float32)
    receive the refined scores; trace ([n, 2 + 2 max_its] float32) and evals
    ([n] int32/uint32) are optional. Device tensors or pointers; asynchronous."""
    n = int(pose_ligand.shape[0]) if hasattr(pose_ligand, "shape") else int(genotypes.shape[0])
    check(lib().dock_local_search(pocket.handle, ligands.handle, C.byref(ls), seed, generation,
                                  _dptr(pose_ligand), n, _dptr(genotypes), _dptr(scores),
                                  _dptr(trace), _dptr(evals), _stream(stream)))


def version() -> str:
    return lib().dock_version().decode()


def dock_features(pocket: Pocket, ligands: Ligands, pose_ligand, genotypes, features, scores=None,
                  stream=None):
    """Features (device uint16/bf16 [n][128]) and optional exact scores of
    genotypes ([n][23] device) posed for ligands pose_ligand ([n] device)."""
    n = int(genotypes.shape[0])
    check(lib().dock_features(pocket.handle, ligands.handle, _dptr(pose_ligand), _dptr(genotypes), n,
                              _dptr(features), _dptr(scores), _stream(stream)))


def dock_features_population(pocket: Pocket, ligands: Ligands, pop: int, genotypes, features,
                             scores=None, stream=None):
    check(lib().dock_features_population(pocket.handle, ligands.handle, pop, _dptr(genotypes),
                                         _dptr(features), _dptr(scores), _stream(stream)))


class Surrogate:
    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            lib().dock_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dock_surrogate_create(seed=0, stream=None) -> Surrogate:
    h = C.c_void_p()
    check(lib().dock_surrogate_create(seed, _stream(stream), C.byref(h)))
    return Surrogate(h)


def dock_surrogate_set_params(s: Surrogate, params, t_mean=0.0, t_std=1.0, t_clip=3.0e38, stream=None):
    p = _c(params, np.float32)
    assert p.shape == (DOCK_MLP_N_PARAMS,)
    check(lib().dock_surrogate_set_params(s.handle, p.ctypes.data_as(C.c_void_p), t_mean, t_std, t_clip,
                                          _stream(stream)))


def dock_surrogate_get_params(s: Surrogate):
    p = np.zeros(DOCK_MLP_N_PARAMS, np.float32)
    m, sd, c = C.c_float(), C.c_float(), C.c_float()
    check(lib().dock_surrogate_get_params(s.handle, p.ctypes.data_as(C.c_void_p), C.byref(m),
                                          C.byref(sd), C.byref(c)))
    return p, m.value, sd.value, c.value


def dock_surrogate_predict(s: Surrogate, features, out, stream=None):
    n = int(features.shape[0])
    check(lib().dock_surrogate_predict(s.handle, _dptr(features), n, _dptr(out), _stream(stream)))


def dock_surrogate_gradients(s: Surrogate, features, targets, grad, stream=None) -> float:
    n = int(features.shape[0])
    loss = C.c_float()
    check(lib().dock_surrogate_gradients(s.handle, _dptr(features), _dptr(targets), n, _dptr(grad),
                                         C.byref(loss), _stream(stream)))
    return loss.value


def dock_surrogate_train(s: Surrogate, features, scores, epochs=2, batch=4096, lr=1e-3,
                         score_clip=20.0, seed=0, stream=None) -> np.ndarray:
    n = int(features.shape[0])
    tp = dock_train_params(epochs, batch, lr, score_clip, seed)
    losses = np.zeros(epochs, np.float32)
    check(lib().dock_surrogate_train(s.handle, _dptr(features), _dptr(scores), n, C.byref(tp),
                                     losses.ctypes.data_as(C.c_void_p), _stream(stream)))
    return losses


def dock_measure_peaks(stream=None):
    """(FP32 FMA TFLOP/s, MUFU ex2 Tops/s) measured on the current device."""
    f, m = C.c_double(), C.c_double()
    check(lib().dock_measure_peaks(C.byref(f), C.byref(m), _stream(stream)))
    return f.value, m.value


def dock_autotune(pocket: Pocket, ligands: Ligands, pop: int, generations: int, seed=0,
                  stream=None, inter=0) -> dict:
    """Measure the search kernel's launch shapes on this ligand set (for the
    inter-energy `inter` names) and keep the fastest for later dock_batch
    calls; returns the measured table."""
    sp = dock_search_params(pop, generations, 0.8, 0.02, seed, 0, 0, 0, None, None,
                            DOCK_MODE_PLAIN, 0, 0, None, dock_ls_params(*NO_LS), None, inter)
    t = dock_tune_table()
    check(lib().dock_autotune(pocket.handle, ligands.handle, C.byref(sp), _stream(stream), C.byref(t)))
    rows = [dict(threads=t.threads[i], atoms_per_lane=t.atoms_per_lane[i],
                 ms_per_generation=t.ms_per_generation[i]) for i in range(t.n)]
    return dict(table=rows, best=t.best)
