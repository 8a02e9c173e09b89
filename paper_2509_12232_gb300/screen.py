"""Chunked screening through the C ABI.

A screen too large for one dock_batch (1,000,000 ligands x 2,048 poses holds
about 110 GB of genotypes per population buffer) is docked in chunks of
ligands. Ligands are independent (the paper docks one ligand per worker,
Section IV), so a chunk's records do not depend on how the screen is cut.
While chunk k is searched on the caller's stream, a host thread prepares
chunk k + 1 (topology, pair lists, records) and uploads it on a second
stream with dock_load_ligands, so the GPU does not wait for host work
between chunks beyond the first. Orchestration only: every step of the
search runs in libdock.
"""
from __future__ import annotations

import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import dock


def _load(pocket, ligs, stream, device):
    if device is not None:
        import torch
        torch.cuda.set_device(device)
    return dock.dock_load_ligands(pocket, ligs.atom_off, ligs.x, ligs.y, ligs.z, ligs.q, ligs.type,
                                  ligs.parent, ligs.tors_off, ligs.tors_b, ligs.ligand_id,
                                  stream=stream)


def screen(pocket, chunks, pop: int, generations: int, seed: int = 0, stream=None,
           side_stream=None, device=None, **search):
    """Dock every ligand of `chunks` (an iterable of ligand sets in host
    arrays, synth.LigandSet fields) with dock_batch(pop, generations, seed,
    **search); returns (records, per-chunk list of (ligands, seconds from
    the chunk's search launch to its records on the host)). The records
    are the dock_result rows of all chunks in order."""
    out, stats = [], []
    it = iter(chunks)
    with ThreadPoolExecutor(1) as ex:
        first = next(it, None)
        nxt = ex.submit(_load, pocket, first, side_stream, device) if first is not None else None
        while nxt is not None:
            gl = nxt.result()
            t0 = time.perf_counter()
            job = dock.dock_batch(pocket, gl, pop, generations, seed=seed, stream=stream, **search)
            ligs = next(it, None)
            nxt = ex.submit(_load, pocket, ligs, side_stream, device) if ligs is not None else None
            out.append(dock.dock_results(job))
            stats.append((gl.n_ligands, time.perf_counter() - t0))
            job.close()
            gl.close()
    recs = np.concatenate(out) if out else np.zeros(0, dock.RESULT_DTYPE)
    return recs, stats
