"""Benchmark of the docking hot path on GB300 (one JSON line on rank 0).

A step is one whole plain-mode search over the batch: every ligand's
population drawn, then (generations - 1) fused GA-step + pose + FP32-score
generations, then the per-ligand best-8 FP64 rescoring, all through the C ABI.
Workload (default): 1,000 synthetic ligands, heavy atoms uniform in 10-60,
rotatable bonds uniform in 0-12, against a 4,000-atom pocket (cavity radius
16 A, 86^3 grid at 0.375 A), 1,024 poses x 50 generations per ligand.

value: ligands/s with the ligand set already resident on the device.
e2e: ligands/s through the public API from host arrays (ligand upload with
its host-side preparation, the search, and the D2H copy of the results), with
batch k + 1 prepared by a second host thread while batch k is searched.
Under torchrun the ranks draw one global set of world x n ligands and each
docks its cost-balanced contiguous range of it (shard.balanced_ranges; weak
scaling, no collective on the data path).

--mode nogrid runs the same plain search with the pairwise inter-energy
(every protein atom within 8 A, no maps) and prints its own line.

--mode lga runs the same workload as the Lamarckian variant (Solis-Wets
refinement of 6% of each generation, at most 300 iterations: AutoDock's
settings) and prints its own line.

--impl reference times the CPU oracle (plain FP64 C, all host cores) on a
bounded sample of the same workload; it is the only other user of oracle/.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c2"
METRIC = "ligands/s (plain exact GA docking: 1,024 poses x 50 generations per ligand)"
DESCR = ("1,000 synthetic ligands (10-60 heavy atoms, 0-12 torsions) vs a 4,000-atom pocket "
         "(16 A cavity, 86^3 x 7 grid maps), 1,024 poses x 50 generations, FP64 best-8 rescoring")
# --workload c3: the uneven batch (one persistent launch per lanes-per-pose
# group and generation, graph-captured, autotuned shape) at its full size
WORKLOADS = {
    "c2": (METRIC, DESCR),
    "c3": ("ligands/s (plain exact GA docking of an uneven batch: 512 poses x 30 generations "
           "per ligand)",
           "100,000 synthetic ligands (heavy atoms lognormal, mean 30, sd 10, clipped to 8-100; "
           "Poisson(5) torsions, at most 16) vs a 4,000-atom pocket (16 A cavity, 86^3 x 7 grid "
           "maps), 512 poses x 30 generations, FP64 best-8 rescoring"),
    "c5": ("ligands/s (plain exact GA docking, large screen in chunks: 2,048 poses x 40 "
           "generations per ligand)",
           "1,000,000 synthetic ligands (10-60 heavy atoms, 0-12 torsions) in 20 chunks of 50,000 "
           "vs a 10,000-atom pocket (20 A cavity, 107^3 x 7 grid maps), 2,048 poses x 40 "
           "generations, FP64 best-8 rescoring"),
}
METRIC_NOGRID = ("ligands/s (plain exact GA docking without grid maps: pairwise inter-energy, "
                 "1,024 poses x 50 generations per ligand)")
METRIC_LGA = ("ligands/s (Lamarckian GA docking: 1,024 poses x 50 generations per ligand, "
              "Solis-Wets on 6% of each generation, up to 300 iterations)")
LS_DEFAULTS = dict(rate=0.06, max_its=300, max_succ=4, max_fail=4, rho=1.0, rho_lb=0.01)

# Algorithmic work per pose (FMA = 2 flops), counted from the operations of
# Algorithms 1 and 2.
FLOP_RIGID_PER_ATOM = 18        # 3x3 rotation + translation
FLOP_POSE_FIXED = 40            # quaternion -> matrix
FLOP_TORSION = 40               # axis, sin/cos, rotation matrix
FLOP_PER_MOVED_ATOM = 21        # rotate one atom about the bond
FLOP_INTER_PER_ATOM = 62        # grid coordinates, 8 corners, 7 lerps
FLOP_PER_PAIR = 34              # distance + the four pair terms + sum
MUFU_PER_PAIR = 4               # rsqrt, 2 x ex2, rcp
MUFU_PER_TORSION = 3            # sin, cos, rsqrt
MUFU_PER_POSE = 1               # rsqrt of the quaternion norm


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def src_hash(files=("search.cu", "pose.cuh", "device_common.cuh", "dock_internal.h")):
    """Hash of the kernel sources a committed ncu summary was taken on."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2509_12232_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


MLP_SOURCES = ("mlp_tc.cu", "mlp.h")


def read_mlp_traffic(rows):
    """DRAM bytes of one fused-forward launch over `rows` feature rows: the
    committed ncu summary's bytes scaled by rows (the features are read once
    and the weights come from L2, so the traffic grows with the rows), if the
    summary was taken on the current kernel source, else None."""
    p = os.path.join(ROOT, "profiles", "mlp_forward_1m.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_hash") != src_hash(MLP_SOURCES):
        return None
    try:
        per_row = (float(kv["dram_bytes_read"]) + float(kv["dram_bytes_write"])) / float(kv["rows"])
    except (KeyError, ValueError):
        return None
    return round(per_row * rows)


def read_profile():
    """key = value pairs of the committed ncu summary of one search generation
    (the search-kernel launches of one generation, one per lanes-per-pose
    group), if it was taken on the current kernel source, else None."""
    p = os.path.join(ROOT, "profiles", "search_kernel_c2.txt")
    if not os.path.exists(p):
        return None
    kv, sect = {}, ""
    for line in open(p):
        line = line.strip()
        if line.startswith("[") and line.endswith("]"):
            sect = line[1:-1] + "."
        elif "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[sect + k.strip()] = v.strip()
    return kv if kv.get("source_hash") == src_hash() else None


def read_issue(per_gen_s, n_sm, sm_mhz):
    """Warp instructions of one generation (ncu summary) over its measured
    time, against the SMs' issue rate (4 schedulers x 1 warp instruction per
    cycle); None when the summary is not of the current source."""
    kv = read_profile()
    if kv is None:
        return None
    try:
        inst = sum(float(v) for k, v in kv.items() if k.endswith(".warp_instructions"))
    except ValueError:
        return None
    peak = n_sm * 4 * sm_mhz * 1e6 / 1e9
    ach = inst / per_gen_s / 1e9
    return {"achieved": round(ach, 1), "peak": round(peak, 1), "unit": "G warp instructions/s",
            "frac": round(ach / peak, 4),
            "source": "ncu warp instructions per generation (profiles/search_kernel_c2.txt) / "
                      "measured generation time"}


def read_traffic():
    """DRAM bytes per search generation (the search-kernel launches of one
    generation, one per lanes-per-pose group) from the committed ncu summary,
    if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "search_kernel_c2.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_hash") != src_hash():
        return None
    try:
        return float(kv["dram_bytes_per_generation"])
    except (KeyError, ValueError):
        return None


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def alu_peaks(dock, stream, n_sm, sm_mhz):
    """(FP32 TFLOP/s, MUFU Tops/s, description): measured on this GPU by
    dock_measure_peaks (independent FMA / ex2 chains on every SM), with the
    unit-count figures (lanes x clock) beside them for reference."""
    f, m = dock.dock_measure_peaks(stream)
    spec_f = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    spec_m = n_sm * 16 * sm_mhz * 1e6 / 1e12
    return f, m, {"peak_source": "measured: dock_measure_peaks (FFMA and ex2 chains on every SM)",
                  "unit_count_peaks": {"fp32_tflops": round(spec_f, 2),
                                       "mufu_tops": round(spec_m, 4),
                                       "from": "%d SMs x 128 FP32 / 16 MUFU lanes x %.0f MHz"
                                               % (n_sm, sm_mhz)}}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def work_per_pose(info, n_lig):
    """Algorithmic FP32 flops and MUFU ops for one pose of every ligand (sum)."""
    flops = (n_lig * FLOP_POSE_FIXED + info["n_atoms"] * (FLOP_RIGID_PER_ATOM + FLOP_INTER_PER_ATOM) +
             info["n_torsions"] * FLOP_TORSION + info["n_moved"] * FLOP_PER_MOVED_ATOM +
             info["n_pairs"] * FLOP_PER_PAIR)
    mufu = n_lig * MUFU_PER_POSE + info["n_torsions"] * MUFU_PER_TORSION + info["n_pairs"] * MUFU_PER_PAIR
    return flops, mufu


def inter_pairs_per_pose(dock, torch, pocket, gl, pk, ligs, w, trace, stream, n=512):
    """Mean number of ligand-protein pairs within 8 A per scored pose of the
    no-grid search: posed coordinates (dock_score) of n poses sampled from
    generation 0 and n from the last generation of a traced search, averaged
    (the count grows as the search moves poses against the protein)."""
    goff = gl.geno_offsets(w.pop)
    tot = int(goff[-1])
    na = np.diff(ligs.atom_off)
    prot = torch.from_numpy(np.stack([pk.x, pk.y, pk.z], 1).astype(np.float32)).cuda()
    rng = np.random.default_rng(11)
    means = []
    for g in (0, w.generations - 1):
        pop = trace[g * tot: (g + 1) * tot]
        lig = rng.integers(0, ligs.n_ligands, n)
        ind = rng.integers(0, w.pop, n)
        genos = torch.zeros((n, 23), dtype=torch.float32, device="cuda")
        for r in range(n):
            G = 7 + ligs.n_tors(int(lig[r]))
            base = int(goff[lig[r]]) + int(ind[r]) * G
            genos[r, :G] = pop[base: base + G]
        coords = torch.zeros((n, 128, 3), dtype=torch.float32, device="cuda")
        sc = torch.zeros(n, dtype=torch.float32, device="cuda")
        dock.dock_score(pocket, gl, torch.from_numpy(lig.astype(np.int32)).cuda(), genos, sc,
                        coords=coords, stream=stream)
        torch.cuda.synchronize()
        cnt = 0
        for r in range(n):
            cnt += int((torch.cdist(coords[r, :int(na[lig[r]])], prot) < 8.0).sum().item())
        means.append(cnt / n)
    return float(np.mean(means))


def reference_sample(ligs, cores, per_core):
    """The fixed CPU sample of a ligand set that both CPU legs time: cores x
    per_core ligands stratified by search cost (the ligand at the middle of
    each of that many equal-count strata of the cost order), listed largest
    first so the oracle's per-ligand work queue balances its threads."""
    from paper_2509_12232_gb300 import shard
    cost = shard.ligand_costs(ligs.atom_off, ligs.tors_off)
    order = np.argsort(cost, kind="stable")
    n = min(ligs.n_ligands, cores * per_core)
    picks = order[((np.arange(n) + 0.5) * ligs.n_ligands / n).astype(np.int64)]
    return [int(i) for i in sorted(picks, key=lambda i: (-cost[i], i))]


def time_oracle(sub, P, pks, grid, w, cores, runs, drop, ls=None):
    """Mean seconds of the kept runs (the first `drop` discarded, as in the
    paper's protocol of ten runs with three dropped)."""
    from oracle import oracle as o
    times = []
    for r in range(runs):
        t0 = time.perf_counter()
        o.dock_batch(sub, P, pks, grid, pop=w.pop, generations=w.generations, seed=0,
                     n_threads=cores, ls=ls)
        if r >= drop:
            times.append(time.perf_counter() - t0)
    return float(np.mean(times)), times


def _oracle_setup():
    from oracle import oracle as o
    from paper_2509_12232_gb300 import synth
    pk, ligs, w = synth.make_workload(WORKLOAD)
    P = o.Params(synth.TYPE_PARAMS)
    pks = o.pocket_from(pk)
    return ligs, w, P, pks, o.grid_build(pks, P)


def run_reference(args, rank, world):
    """CPU oracle on the host cores: each step docks the fixed stratified
    sample (reference_sample); warm-up steps are dropped."""
    if rank != 0:
        return 0
    ligs, w, P, pks, grid = _oracle_setup()
    cores = os.cpu_count() or 1
    idx = reference_sample(ligs, cores, args.ref_ligands_per_core)
    sub = ligs.subset(idx)
    mean_s, times = time_oracle(sub, P, pks, grid, w, cores, args.warmup + args.steps, args.warmup)
    value = len(idx) / mean_s
    sample = ("%d ligands (%d per core, stratified by cost) of the %s set, full %d poses x %d "
              "generations each, every step; mean of %d steps after %d dropped" % (
                  len(idx), args.ref_ligands_per_core, WORKLOAD, w.pop, w.generations, len(times),
                  args.warmup))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ligands/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * mean_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": DESCR, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "ligands/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "ligands/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(per_core, lga=False):
    """The oracle as it stands, on all host cores, on the same fixed sample as
    the reference arm: ten runs, the first three dropped (the paper's
    protocol); lga: the Lamarckian variant."""
    from oracle import oracle as o
    ligs, w, P, pks, grid = _oracle_setup()
    cores = os.cpu_count() or 1
    ls = o.LsParams(**LS_DEFAULTS) if lga else None
    # the Lamarckian oracle scores ~10x more poses per ligand: one ligand per
    # core and two runs (one dropped) keep it within the bench's minutes
    per_core, runs, drop = (1, 2, 1) if lga else (per_core, 10, 3)
    idx = reference_sample(ligs, cores, per_core)
    mean_s, times = time_oracle(ligs.subset(idx), P, pks, grid, w, cores, runs, drop, ls=ls)
    return {"value": len(idx) / mean_s, "unit": "ligands/s", "cores": cores, "kind": "oracle",
            "sample": "%d ligands (%d per core, stratified by cost) of the %s set, full %d poses x "
                      "%d generations each; mean of %d runs after %d dropped, %.2f s per run" % (
                          len(idx), per_core, WORKLOAD, w.pop, w.generations, runs - drop, drop,
                          mean_s)}


def _make_chunk(args):
    from paper_2509_12232_gb300 import synth
    name, c, size = args
    return synth.screen_chunk(name, c, size)


def run_screen(args, rank, world):
    """The large screen (c5): every chunk docked through the C ABI from host
    arrays, chunk k + 1 prepared and uploaded on a side stream while chunk k
    is searched (screen.screen). The ligands are drawn before the timed
    region, in parallel processes; the timed region covers the whole screen
    (upload, search, FP64 rescoring, records to the host)."""
    import multiprocessing as mp
    from paper_2509_12232_gb300 import synth
    size = args.screen_chunk
    w = synth.WORKLOADS[WORKLOAD]
    n_total = args.ligands or w.n_ligands
    n_chunks = -(-n_total // size)
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(n_chunks, os.cpu_count() or 1)) as pool:
        chunks = pool.map(_make_chunk, [(WORKLOAD, c, size) for c in range(n_chunks)])
    if n_total % size:
        chunks[-1] = chunks[-1].subset(np.arange(n_total - (n_chunks - 1) * size))
    gen_s = time.perf_counter() - t0
    import torch
    from paper_2509_12232_gb300 import build, dock, screen
    torch.cuda.set_device(0)
    build.build()
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    pk, _, _ = synth.make_workload(WORKLOAD, n_ligands=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pocket = dock.dock_create_pocket(pk.x, pk.y, pk.z, pk.q, pk.type, pk.center, pk.radius,
                                     pk.spacing, synth.TYPE_PARAMS, stream=stream)
    torch.cuda.synchronize()
    grid_ms = 1000 * (time.perf_counter() - t0)
    # set-up (untimed): launch shape measured on 2,000 ligands of chunk 0,
    # then kept for every chunk; one profiled search of them for the roofline
    probe = chunks[0].subset(np.arange(min(2000, chunks[0].n_ligands)))
    gp = screen._load(pocket, probe, stream, None)
    tune = dock.dock_autotune(pocket, gp, w.pop, 4, stream=stream)
    shape = tune["table"][tune["best"]]
    os.environ["DOCK_THREADS"] = str(shape["threads"])
    os.environ["DOCK_ATOMS_PER_LANE"] = str(shape["atoms_per_lane"])
    info = dock.dock_ligands_info(gp)
    os.environ["DOCK_PROFILE_LAUNCHES"] = "1"
    j = dock.dock_batch(pocket, gp, w.pop, w.generations, seed=0, use_graph=1, stream=stream)
    ms_kernels, n_launch = dock.dock_job_kernel_time(j)
    dock.dock_results(j)
    j.close()
    del os.environ["DOCK_PROFILE_LAUNCHES"]
    gp.close()
    clocks = Clocks(0)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    recs, stats = screen.screen(pocket, chunks, w.pop, w.generations, seed=0, stream=stream,
                                side_stream=side, device=0, use_graph=1)
    torch.cuda.synchronize()
    total_s = time.perf_counter() - t0
    clk = clocks.stop()
    assert recs.shape[0] == n_total and np.all(recs["status"] == 0)
    assert np.array_equal(recs["ligand_id"], np.arange(n_total, dtype=np.uint64))
    peaks, _ = measured_peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak, mufu_peak, peak_src = alu_peaks(dock, stream, n_sm, sm_mhz)
    flops_pose, mufu_pose = work_per_pose(info, probe.n_ligands)
    per_gen_s = ms_kernels / 1000.0 / max(n_launch, 1)
    ach = flops_pose * w.pop / per_gen_s / 1e12
    poses = n_total * w.pop * w.generations
    line = {"metric": METRIC, "value": round(n_total / total_s, 2), "unit": "ligands/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": round(1000 * total_s, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": DESCR, "ligands": n_total, "chunk": size, "chunks": n_chunks,
                       "pop": w.pop, "generations": w.generations,
                       "l2": "inputs larger than L2 (each chunk's genotypes ~10 GB)",
                       "launch_shape": {"threads": shape["threads"],
                                        "atoms_per_lane": shape["atoms_per_lane"],
                                        "picked_by": "dock_autotune on 2,000 ligands of chunk 0"}},
            "poses_scored_per_s": round(poses / total_s, 1),
            "timed_region": "whole screen from host ligand arrays: per chunk upload (overlapped "
                            "with the previous chunk's search), search, FP64 rescoring, records "
                            "to the host",
            "chunk_seconds": {"min": round(min(t for _, t in stats), 3),
                              "max": round(max(t for _, t in stats), 3)},
            "roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": round(fp32_peak, 2),
                         "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4), "traffic": None,
                         "kernel": "search_kernel", **peak_src,
                         "measured_on": "one profiled search of 2,000 ligands of chunk 0",
                         "mufu": {"achieved": round(mufu_pose * w.pop / per_gen_s / 1e12, 4),
                                  "peak": round(mufu_peak, 4), "unit": "Tops/s",
                                  "frac": round(mufu_pose * w.pop / per_gen_s / 1e12 / mufu_peak,
                                                4)},
                         "generation_ms": round(1000 * per_gen_s, 4)},
            "grid_build_ms": round(grid_ms, 1), "ligand_generation_s (untimed)": round(gen_s, 1),
            "gpu_launches": n_chunks * (n_launch + 4),
            "gpu_launches_note": "per chunk: the search launches of 40 generations (as counted in "
                                 "the profiled search) plus the set-up and FP64 rescoring kernels",
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_fp32(per_core):
    """The paper's own style of CPU hot path (oracle/simd_fp32.c: FP32 SoA
    loops auto-vectorised with #pragma omp simd, -O3 -ffast-math, one ligand
    per thread) on the same sample and protocol as cpu_baseline: context, a
    fairer CPU reference point than the FP64 oracle."""
    from oracle import oracle as o
    ligs, w, P, pks, grid = _oracle_setup()
    cores = os.cpu_count() or 1
    sub = ligs.subset(reference_sample(ligs, cores, per_core))
    times = []
    for r in range(10):
        t0 = time.perf_counter()
        o.cpu32_dock_batch(sub, P, pks, grid, w.pop, w.generations, seed=0, n_threads=cores)
        if r >= 3:
            times.append(time.perf_counter() - t0)
    mean_s = float(np.mean(times))
    return {"value": sub.n_ligands / mean_s, "unit": "ligands/s", "cores": cores,
            "kind": "fp32-simd (the paper's auto-vectorised CPU style; no FP64 rescoring)",
            "sample": "the cpu_baseline sample (%d ligands); mean of 7 runs after 3 dropped, "
                      "%.2f s per run" % (sub.n_ligands, mean_s)}


def run_surrogate(args, rank, world):
    """Surrogate-pre-screened vs plain exact search on the same GPU and ligands
    (large-screen per-ligand settings: c2 size mix, 10,000-atom pocket,
    2,048 poses x 40 generations, 4,096 candidates, 410 kept), on a sample of
    args.ligands ligands. Training (per pocket, on ~10M exact pairs of
    training ligands drawn with another seed) is timed separately."""
    import torch
    from paper_2509_12232_gb300 import build, dock, synth
    torch.cuda.set_device(local_rank := env_rank()[2])
    build.build()
    stream = torch.cuda.current_stream()
    w = synth.WORKLOADS["c5"]
    pk = synth.make_pocket(w.pocket_atoms, w.radius, seed=0)
    pocket = dock.dock_create_pocket(pk.x, pk.y, pk.z, pk.q, pk.type, pk.center, pk.radius,
                                     pk.spacing, synth.TYPE_PARAMS, stream=stream)

    def ligand_set(n, seed, id_base):
        rng = np.random.Generator(np.random.Philox(seed))
        na, nt = synth.ligand_sizes(rng, "uniform", n)
        ls = synth.make_ligands(rng, na, nt, id_base=id_base)
        return ls, dock.dock_load_ligands(pocket, ls.atom_off, ls.x, ls.y, ls.z, ls.q, ls.type,
                                          ls.parent, ls.tors_off, ls.tors_b, ls.ligand_id,
                                          stream=stream)
    # training pairs: every pose of plain GA trajectories of training ligands
    t0 = time.perf_counter()
    n_tr, pop_tr, gens_tr = 512, 1024, 20
    _, gl_tr = ligand_set(n_tr, 7777, 10 ** 7)
    goff = gl_tr.geno_offsets(pop_tr)
    tot = int(goff[-1])
    tg = torch.zeros(gens_tr * tot, dtype=torch.float32, device="cuda")
    job = dock.dock_batch(pocket, gl_tr, pop_tr, gens_tr, seed=1, trace_genotypes=tg, stream=stream)
    dock.dock_results(job)
    rows = n_tr * pop_tr
    F = torch.zeros(gens_tr * rows, 128, dtype=torch.int16, device="cuda")
    Y = torch.zeros(gens_tr * rows, dtype=torch.float32, device="cuda")
    for g in range(gens_tr):
        dock.dock_features_population(pocket, gl_tr, pop_tr, tg[g * tot:(g + 1) * tot],
                                      F[g * rows:(g + 1) * rows], Y[g * rows:(g + 1) * rows])
    del tg
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    S = dock.dock_surrogate_create(seed=2)
    t0 = time.perf_counter()
    losses = dock.dock_surrogate_train(S, F, Y, epochs=3, batch=4096, lr=1e-3, score_clip=100.0)
    t_train = time.perf_counter() - t0
    del F, Y
    # evaluation ligands
    n = args.ligands or 1000
    ls, gl = ligand_set(n, 1000, 0)
    common = dict(seed=0, stream=stream)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            j = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1000.0, j
    plain_s, jp = timed(lambda: dock.dock_batch(pocket, gl, w.pop, w.generations, **common), args.steps)
    rp = dock.dock_results(jp)
    sur_s, js = timed(lambda: dock.dock_batch(pocket, gl, w.pop, w.generations, surrogate=S,
                                              candidates=2 * w.pop, keep=410, **common), args.steps)
    rs = dock.dock_results(js)
    diff = rs["best_fp64"][:, 0] - rp["best_fp64"][:, 0]
    # the criterion's floor: the same plain search with another seed lands on
    # another best pose; no search whose trajectory differs from the plain
    # one's (any pre-screen does) can be expected to agree more closely
    jq = dock.dock_batch(pocket, gl, w.pop, w.generations, seed=1, stream=stream)
    rq = dock.dock_results(jq)
    floor = rq["best_fp64"][:, 0] - rp["best_fp64"][:, 0]
    line = {"metric": "ligands/s, surrogate-pre-screened GA vs plain exact GA (2,048 poses x 40 "
                      "generations; 4,096 candidates per generation, 410 scored exactly)",
            "value": round(n / sur_s, 2), "unit": "ligands/s", "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": round(sur_s * 1000, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
            "config": {"workload": "%d ligands (10-60 atoms, 0-12 torsions) vs a 10,000-atom pocket "
                                   "(20 A cavity, 107^3 grid)" % n},
            "plain_ligands_per_s": round(n / plain_s, 2),
            "surrogate_over_plain": round(plain_s / sur_s, 3),
            "top1_fp64_surrogate_minus_plain": {
                "median": round(float(np.median(diff)), 4),
                "frac_within_0.1": round(float(np.mean(np.abs(diff) <= 0.1)), 4),
                "frac_surrogate_better_or_within_0.1": round(float(np.mean(diff <= 0.1)), 4)},
            "top1_fp64_plain_seed1_minus_plain_seed0": {
                "median": round(float(np.median(floor)), 4),
                "median_abs": round(float(np.median(np.abs(floor))), 4),
                "frac_within_0.1": round(float(np.mean(np.abs(floor) <= 0.1)), 4)},
            "exact_evals_per_ligand": {"plain": int(rp["exact_evals"][0]),
                                       "surrogate": int(rs["exact_evals"][0])},
            "surrogate_evals_per_ligand": int(rs["surrogate_evals"][0]),
            "training": {"pairs": gens_tr * rows, "data_seconds": round(t_data, 2),
                         "train_seconds": round(t_train, 2),
                         "loss_per_epoch": [round(float(x), 4) for x in losses]}}
    print(json.dumps(line), flush=True)
    return 0


def run_mlp(args, rank, world):
    """The surrogate network alone: the fused tensor-core forward pass over one
    pre-screened generation's candidates (1,000 ligands x 4,096 = 4,194,304
    feature rows), against the measured BF16 peak; and the training step
    (forward, backward, Adam) over 2,097,152 rows in batches of 4,096."""
    import torch
    from paper_2509_12232_gb300 import build, dock
    torch.cuda.set_device(env_rank()[2])
    build.build()
    stream = torch.cuda.current_stream()
    S = dock.dock_surrogate_create(seed=2)
    rows = args.ligands * 4096 if args.ligands else 4 << 20
    g = torch.Generator(device="cuda").manual_seed(7)
    X = (torch.randn(rows, 128, device="cuda", generator=g) * 0.5).to(torch.bfloat16).view(torch.int16)
    out = torch.empty(rows, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        dock.dock_surrogate_predict(S, X, out)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        dock.dock_surrogate_predict(S, X, out)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    flops_row = 2 * (128 * 256 + 2 * 256 * 256 + 256)
    peaks, peak_kind = measured_peaks()
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    ach = flops_row * rows / (ms / 1000.0) / 1e12
    n_tr = 2 << 20
    Y = torch.randn(n_tr, device="cuda", generator=g)
    # training throughput by batch size: a step is a dozen dependent small
    # launches, so small batches are bound by the chain, large ones by the products
    by_batch = {}
    for b in (4096, 16384, 65536):
        dock.dock_surrogate_train(S, X[:n_tr], Y, epochs=1, batch=b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dock.dock_surrogate_train(S, X[:n_tr], Y, epochs=2, batch=b)
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / 2
        by_batch[b] = {"s_per_epoch": round(sec, 4), "us_per_step": round(sec / (n_tr // b) * 1e6, 1),
                       "tflops": round(3 * flops_row * n_tr / sec / 1e12, 2)}
    tr_s = by_batch[4096]["s_per_epoch"]
    line = {"metric": "surrogate candidates predicted per s (fused tensor-core forward pass, "
                      "128-256-256-256-1 BF16 MLP)",
            "value": round(rows / (ms / 1000.0), 1), "unit": "rows/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": "%d BF16 feature rows (one pre-screened generation of %d "
                                   "ligands x 4,096 candidates)" % (rows, rows // 4096),
                       "l2": "flushed between steps (256 MiB write)"},
            "roofline": {"bound": "tensor", "achieved": round(ach, 2), "peak": bf16,
                         "unit": "TFLOP/s", "frac": round(ach / bf16, 4),
                         "traffic": read_mlp_traffic(rows),
                         "kernel": "fused_forward_kernel",
                         "peak_source": "bf16_tflops (%s)" % peak_kind},
            "training": {"rows_per_epoch": n_tr, "batch": 4096, "s_per_epoch": round(tr_s, 4),
                         "tflops": round(3 * flops_row * n_tr / tr_s / 1e12, 2),
                         "by_batch": by_batch}}
    print(json.dumps(line), flush=True)
    return 0


def run_grid(args, rank, world):
    """The per-pocket grid-map build (the AutoGrid step, timed apart from the
    search): dock_create_pocket end to end (host cell list and tables, device
    allocations, the map kernel, the scorer's record layout) for the c2 pocket
    (4,000 atoms, 86^3 nodes x 7 types) and the c5 pocket (10,000 atoms,
    107^3 nodes)."""
    import torch
    from paper_2509_12232_gb300 import build, dock, synth
    torch.cuda.set_device(env_rank()[2])
    build.build()
    out = {}
    for name in ("c2", "c5"):
        w = synth.WORKLOADS[name]
        pk = synth.make_pocket(w.pocket_atoms, w.radius, seed=0)
        make = lambda: dock.dock_create_pocket(pk.x, pk.y, pk.z, pk.q, pk.type, pk.center,  # noqa
                                               pk.radius, pk.spacing, synth.TYPE_PARAMS)
        for _ in range(args.warmup):
            make().close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            make().close()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / args.steps * 1e3
        n = int(round(2 * w.radius / pk.spacing)) + 1
        out[name] = {"atoms": w.pocket_atoms, "nodes": n ** 3, "types": synth.N_TYPES,
                     "ms_per_pocket": round(ms, 3),
                     "node_types_per_s": round(n ** 3 * synth.N_TYPES / (ms / 1000.0), 1)}
    line = {"metric": "pocket grid builds per s (dock_create_pocket, c2 pocket)",
            "value": round(1000.0 / out["c2"]["ms_per_pocket"], 3), "unit": "pockets/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["c2"]["ms_per_pocket"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "grid maps of the c2 and c5 pockets", "pockets": out},
            "roofline": None}
    print(json.dumps(line), flush=True)
    return 0


def run_pairwise(args, rank, world):
    """Pairwise inter-energy scoring without maps (dock_score_pairwise): every
    protein atom within 8 A of each ligand atom enters through the pair
    terms, plus the intra-energy. c2 pocket and ligand set, 256 random poses
    per ligand (256,000 poses per step) with translations in the cavity."""
    import torch
    from paper_2509_12232_gb300 import build, dock, synth
    local = env_rank()[2]
    torch.cuda.set_device(local)
    build.build()
    dock.lib()
    stream = torch.cuda.current_stream()
    pk, ligs, w = synth.make_workload(WORKLOAD, pocket=True)
    pocket = dock.dock_create_pocket(pk.x, pk.y, pk.z, pk.q, pk.type, pk.center, pk.radius,
                                     pk.spacing, synth.TYPE_PARAMS, stream=stream)
    largs = (ligs.atom_off, ligs.x, ligs.y, ligs.z, ligs.q, ligs.type, ligs.parent, ligs.tors_off,
             ligs.tors_b, ligs.ligand_id)
    gl = dock.dock_load_ligands(pocket, *largs, stream=stream)
    info = dock.dock_ligands_info(gl)
    per = 256
    nl = ligs.n_ligands
    n = nl * per
    rng = np.random.default_rng(7)
    g = np.zeros((n, 23), np.float32)
    g[:, :3] = rng.uniform(-0.5, 0.5, (n, 3)) * pk.radius
    q = rng.normal(size=(n, 4))
    g[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
    g[:, 7:] = rng.uniform(-np.pi, np.pi, (n, 16))
    pl = np.repeat(np.arange(nl, dtype=np.int32), per)
    dg = torch.from_numpy(g).cuda()
    dpl = torch.from_numpy(pl).cuda()
    sc = torch.zeros(n, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        dock.dock_score_pairwise(pocket, gl, dpl, dg, sc, stream=stream)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        dock.dock_score_pairwise(pocket, gl, dpl, dg, sc, stream=stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_step = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    value = n / (ms_step / 1000.0)
    # algorithmic work: the pose and intra pairs as in the grid scorer, plus every
    # ligand-protein pair within the cutoff (34 flops, 4 MUFU each); the pairs
    # within the cutoff are counted on 1,024 sampled poses (posed by dock_score)
    idx = np.linspace(0, n - 1, 1024).astype(np.int64)
    sub_g, sub_l = dg[idx].contiguous(), dpl[idx].contiguous()
    coords = torch.zeros((len(idx), 128, 3), dtype=torch.float32, device="cuda")
    tmp = torch.zeros(len(idx), dtype=torch.float32, device="cuda")
    dock.dock_score(pocket, gl, sub_l, sub_g, tmp, coords=coords, stream=stream)
    torch.cuda.synchronize()
    prot = torch.from_numpy(np.stack([pk.x, pk.y, pk.z], 1).astype(np.float32)).cuda()
    na = np.diff(ligs.atom_off)
    inter_pairs = 0
    for j, p in enumerate(idx.tolist()):
        x = coords[j, :int(na[pl[p]])]
        inter_pairs += int((torch.cdist(x, prot) < 8.0).sum().item())
    inter_per_pose = inter_pairs / len(idx)
    flops_pose, mufu_pose = work_per_pose(info, nl)
    base = (flops_pose - info["n_atoms"] * FLOP_INTER_PER_ATOM) / nl
    flops = n * (base + inter_per_pose * FLOP_PER_PAIR)
    mufu = n * (mufu_pose / nl + inter_per_pose * MUFU_PER_PAIR)
    peaks, peak_kind = measured_peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak, mufu_peak, peak_src = alu_peaks(dock, stream, n_sm, sm_mhz)
    ach = flops / (ms_step / 1000.0) / 1e12
    achm = mufu / (ms_step / 1000.0) / 1e12
    # end to end from host genotypes: upload, score, download
    hg = torch.from_numpy(g).pin_memory()
    hs = torch.zeros(n, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dg.copy_(hg, non_blocking=True)
        dock.dock_score_pairwise(pocket, gl, dpl, dg, sc, stream=stream)
        hs.copy_(sc, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    line = {"metric": "poses/s (pairwise inter-energy + intra-energy scoring, no grid maps)",
            "value": round(value, 1), "unit": "poses/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c2 pocket (4,000 atoms) and ligand set, 256 random poses per "
                                   "ligand (%d poses)" % n,
                       "l2": "flushed between steps (256 MiB write)",
                       "protein_pairs_within_cutoff_per_pose": round(inter_per_pose, 1)},
            "roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": round(fp32_peak, 2),
                         "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4), "traffic": None,
                         "kernel": "score_pairwise_kernel", **peak_src,
                         "mufu": {"achieved": round(achm, 4), "peak": round(mufu_peak, 4),
                                  "unit": "Tops/s", "frac": round(achm / mufu_peak, 4)}},
            "e2e": {"value": round(n / e2e_s, 1), "unit": "poses/s",
                    "h2d_bytes_per_step": int(g.nbytes), "d2h_bytes_per_step": int(n * 4)},
            "gpu_launches": args.steps, "clocks": clk}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = pairwise_cpu_baseline(ligs, pk, g, pl, args.cpu_baseline_seconds)
    print(json.dumps(line), flush=True)
    return 0


def pairwise_cpu_baseline(ligs, pk, g, pl, budget_s):
    """The oracle's pairwise score (FP64 C, one core) on the first poses of
    the same set, about budget_s seconds."""
    from oracle import oracle as o
    from paper_2509_12232_gb300 import synth
    P = o.Params(synth.TYPE_PARAMS)
    pks = o.pocket_from(pk)
    lig_cache = {}
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s and done < len(pl):
        l = int(pl[done])
        if l not in lig_cache:
            lig_cache[l] = o.Ligand(**ligs.ligand(l))
        lig = lig_cache[l]
        xyz = o.pose(lig, g[done, :lig.n_genes], pk.center)
        o.inter_pairwise(lig, P, pks, xyz)
        o.intra(lig, P, xyz)
        done += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "poses/s", "cores": 1, "kind": "oracle",
            "sample": "first %d poses of the same set, %.1f s" % (done, dt)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="plain",
                    choices=["plain", "lga", "nogrid", "surrogate", "mlp", "grid", "pairwise"],
                    help="lga: the Lamarckian search (Solis-Wets); surrogate: pre-screened vs "
                         "plain comparison; mlp: the surrogate network's forward pass and training "
                         "step alone; grid: the pocket grid build (each its own JSON line)")
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS),
                    help="c2 (default): 1,000 ligands x 1,024 poses x 50 generations; c3: the "
                         "uneven batch, 100,000 ligands x 512 poses x 30 generations "
                         "(plain, lga and nogrid modes); c5: the large screen, 1,000,000 "
                         "ligands x 2,048 poses x 40 generations in chunks (plain)")
    ap.add_argument("--screen-chunk", type=int, default=50_000,
                    help="ligands per dock_batch call of the c5 screen")
    ap.add_argument("--ref-ligands-per-core", type=int, default=2)
    ap.add_argument("--cpu-baseline-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ligands", type=int, default=0,
                    help="dock only the first N ligands (profiling runs; not a bench line)")
    ap.add_argument("--shape", default="",
                    help="THREADSxATOMS_PER_LANE launch shape instead of dock_autotune's pick "
                         "(profiling runs)")
    args = ap.parse_args()
    global WORKLOAD, METRIC, DESCR
    WORKLOAD = args.workload
    METRIC, DESCR = WORKLOADS[WORKLOAD]
    rank, world, local = env_rank()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.mode == "surrogate":
        return run_surrogate(args, rank, world)
    if args.mode == "mlp":
        return run_mlp(args, rank, world)
    if args.mode == "grid":
        return run_grid(args, rank, world)
    if args.mode == "pairwise":
        return run_pairwise(args, rank, world)
    if WORKLOAD == "c5":
        return run_screen(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2509_12232_gb300 import build, dock, synth

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    build.build()
    dock.lib()
    stream = torch.cuda.current_stream()
    pk, _, w = synth.make_workload(WORKLOAD, pocket=True)
    # one global set of world x n ligands (weak scaling: n per GPU), drawn the
    # same way on every rank; rank r docks the r-th cost-balanced contiguous
    # range of it (no collective on the data path)
    rng = np.random.Generator(np.random.Philox(1000))
    if args.ligands:
        w.n_ligands = args.ligands
    n_global = w.n_ligands * world
    na, nt = synth.ligand_sizes(rng, w.sizes, n_global)
    ligs = synth.make_ligands(rng, na, nt, id_base=0)
    if world > 1:
        from paper_2509_12232_gb300 import shard
        a, b = shard.balanced_ranges(shard.ligand_costs(ligs.atom_off, ligs.tors_off), world)[rank]
        ligs = ligs.subset(np.arange(a, b))
    pocket = dock.dock_create_pocket(pk.x, pk.y, pk.z, pk.q, pk.type, pk.center, pk.radius,
                                     pk.spacing, synth.TYPE_PARAMS, stream=stream)
    largs = (ligs.atom_off, ligs.x, ligs.y, ligs.z, ligs.q, ligs.type, ligs.parent, ligs.tors_off,
             ligs.tors_b, ligs.ligand_id)
    gl = dock.dock_load_ligands(pocket, *largs, stream=stream)
    info = dock.dock_ligands_info(gl)
    # launch shape of the search kernel: measured on this ligand set (set-up, not timed)
    if args.shape:
        t_, a_ = (int(v) for v in args.shape.lower().split("x"))
        shape = {"threads": t_, "atoms_per_lane": a_}
        os.environ["DOCK_THREADS"], os.environ["DOCK_ATOMS_PER_LANE"] = str(t_), str(a_)
        picked_by = "--shape"
    else:
        tune = dock.dock_autotune(pocket, gl, w.pop, 4, stream=stream,
                                  inter=dock.DOCK_INTER_PAIRWISE if args.mode == "nogrid"
                                  else dock.DOCK_INTER_GRID)
        shape = tune["table"][tune["best"]]
        picked_by = "dock_autotune"
    # one search launch per lanes-per-pose group L (smallest L in 1, 2, 4, 8
    # with L * atoms_per_lane >= atoms) and generation
    apl = shape["atoms_per_lane"]
    groups = sorted({next(L for L in (1, 2, 4, 8) if L * apl >= n or L == 8)
                     for n in np.diff(ligs.atom_off)})
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    lga = args.mode == "lga"
    nogrid = args.mode == "nogrid"
    ls = dock.ls_params(**LS_DEFAULTS) if lga else None
    inter = dock.DOCK_INTER_PAIRWISE if nogrid else dock.DOCK_INTER_GRID

    def step(**kw):
        job = dock.dock_batch(pocket, gl, w.pop, w.generations, seed=0, use_graph=1, stream=stream,
                              ls=ls, inter=inter, **kw)
        return job

    # warm-up
    for _ in range(args.warmup):
        j = step()
        torch.cuda.synchronize()
        j.close()
    # per-launch kernel times for the roofline (separate profiled pass); in
    # the Lamarckian search also the scorings per ligand (GA + local search)
    os.environ["DOCK_PROFILE_LAUNCHES"] = "1"
    trace = None
    if nogrid:  # populations of every generation, for the pair count below
        trace = torch.zeros(w.generations * int(gl.geno_offsets(w.pop)[-1]), dtype=torch.float32,
                            device="cuda")
    j = step(trace_genotypes=trace)
    ms_kernels, n_launch = dock.dock_job_kernel_time(j)
    evals_total = int(dock.dock_results(j)["exact_evals"].sum())
    j.close()
    del os.environ["DOCK_PROFILE_LAUNCHES"]
    inter_per_pose = None
    if nogrid:
        inter_per_pose = inter_pairs_per_pose(dock, torch, pocket, gl, pk, ligs, w, trace, stream)
        del trace
    # timed region
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    jobs = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)          # evict L2 between steps
        ev[i][0].record(stream)
        jobs.append(step())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    for j in jobs:
        j.close()
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    ms_step = ms / args.steps
    total_ligands = n_global
    value = total_ligands / (ms_step / 1000.0)
    poses_per_step = n_global * w.pop * w.generations

    # end to end through the public API from host arrays, as a screening run
    # streams its batches: a second host thread prepares and uploads batch
    # k + 1 (dock_load_ligands on a side stream) while batch k is searched,
    # and batch k's results are read once batch k + 1 is queued behind it, so
    # the GPU does not idle while the host reads results and enqueues. The
    # ligand sets are destroyed after the last results (freeing device memory
    # waits for the whole device to drain); the first batch's preparation
    # (pipeline fill), the last batch's results and the destroys are inside
    # the timed region
    h2d = info["h2d_bytes"]
    d2h = ligs.n_ligands * dock.RESULT_DTYPE.itemsize + 4
    side = torch.cuda.Stream()

    def load():
        torch.cuda.set_device(local)
        return dock.dock_load_ligands(pocket, *largs, stream=side)

    torch.cuda.synchronize()
    with ThreadPoolExecutor(1) as ex:
        t0 = time.perf_counter()
        nxt = ex.submit(load)
        prev, sets = None, []
        for i in range(args.e2e_steps):
            g2 = nxt.result()
            sets.append(g2)
            j = dock.dock_batch(pocket, g2, w.pop, w.generations, seed=0, use_graph=1,
                                stream=stream, ls=ls, inter=inter)
            if i + 1 < args.e2e_steps:
                nxt = ex.submit(load)
            if prev is not None:
                dock.dock_results(prev)
                prev.close()
            prev = j
        if prev is not None:
            dock.dock_results(prev)
            prev.close()
        for g2 in sets:
            g2.close()
        e2e_s = (time.perf_counter() - t0) / max(args.e2e_steps, 1)
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    if rank != 0:
        dist.destroy_process_group()
        return 0
    peaks, peak_kind = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak, mufu_peak, peak_src = alu_peaks(dock, stream, n_sm, sm_mhz)  # TFLOP/s, Tops/s
    flops_pose, mufu_pose = work_per_pose(info, ligs.n_ligands)
    per_gen_s = ms_kernels / 1000.0 / max(n_launch, 1)
    # poses scored per generation per ligand: pop (GA), plus in the Lamarckian
    # search the local-search probes (the mean per-pose work of the set)
    poses_gen = w.pop if not lga else evals_total / ligs.n_ligands / w.generations
    if nogrid:
        # no grid lookups; every ligand-protein pair within the cutoff instead
        flops_pose += ligs.n_ligands * inter_per_pose * FLOP_PER_PAIR - info["n_atoms"] * FLOP_INTER_PER_ATOM
        mufu_pose += ligs.n_ligands * inter_per_pose * MUFU_PER_PAIR
    ach_fp32 = flops_pose * poses_gen / per_gen_s / 1e12
    ach_mufu = mufu_pose * poses_gen / per_gen_s / 1e12
    roof = {"bound": "alu", "achieved": round(ach_fp32, 3), "peak": round(fp32_peak, 2),
            "unit": "TFLOP/s", "frac": round(ach_fp32 / fp32_peak, 4),
            "traffic": None if (lga or nogrid or WORKLOAD != "c2") else read_traffic(),
            "kernel": ("search_kernel + ls_kernel" if lga else
                       "search_kernel<L, pairwise>" if nogrid else "search_kernel"),
            **peak_src,
            "mufu": {"achieved": round(ach_mufu, 4), "peak": round(mufu_peak, 4), "unit": "Tops/s",
                     "frac": round(ach_mufu / mufu_peak, 4)},
            "issue": None if (lga or nogrid or WORKLOAD != "c2") else read_issue(per_gen_s, n_sm,
                                                                                 sm_mhz),
            "generation_ms": round(per_gen_s * 1000, 4), "generations_timed": n_launch,
            "launches_per_generation": len(groups), "lanes_per_pose_groups": groups}
    metric = METRIC_LGA if lga else METRIC_NOGRID if nogrid else METRIC
    metric = metric.replace("1,024 poses x 50 generations",
                            "{:,} poses x {} generations".format(w.pop, w.generations))
    line = {"metric": metric,
            "value": round(value, 2), "unit": "ligands/s",
            "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": DESCR, "l2": "flushed between steps (256 MiB write)",
                       "ligands_per_gpu": w.n_ligands, "pop": w.pop, "generations": w.generations,
                       "launch_shape": {"threads": shape["threads"],
                                        "atoms_per_lane": shape["atoms_per_lane"],
                                        "picked_by": picked_by}},
            "poses_scored_per_s": round((evals_total * world if lga else poses_per_step) /
                                        (ms_step / 1000.0), 1),
            "roofline": roof,
            "e2e": {"value": round(total_ligands / e2e_s, 2), "unit": "ligands/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "steps": args.e2e_steps,
                    "pipeline": "batch k+1 prepared and uploaded by a second host thread "
                                "while batch k is searched; batch k's results read once batch "
                                "k+1 is queued; ligand sets destroyed after the last results; "
                                "first preparation, last results and destroys included"},
            "gpu_launches": args.steps * (w.generations * len(groups) * (2 if lga else 1) + 1),
            "clocks": clk}
    if nogrid:
        line["config"]["protein_pairs_within_cutoff_per_pose"] = round(inter_per_pose, 1)
        line["config"]["inter"] = "pairwise over a protein cell list (8 A rows in y-z, 1 A cells in x, rows trimmed to the cutoff chord; no maps)"
    if lga:
        line["config"]["local_search"] = dict(LS_DEFAULTS, method="Solis-Wets, Lamarckian")
        line["scorings_per_step"] = evals_total * world
    if not args.no_cpu_baseline and world == 1 and not nogrid:
        line["cpu_baseline"] = cpu_baseline(args.ref_ligands_per_core, lga=lga)
        if not lga:
            line["cpu_baseline_fp32_simd"] = cpu_baseline_fp32(args.ref_ligands_per_core)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
