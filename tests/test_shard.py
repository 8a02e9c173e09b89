"""Multi-process sharding of ligands (gloo, world size 2, CPU): the ranks'
contiguous ranges cover the batch exactly once and balance the cost; each
rank docks its range with the FP64 oracle, the per-ligand result records are
gathered with shard.gather_records and must equal, bit for bit, one
single-process docking of the whole batch; the step time is the maximum
over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2509_12232_gb300 import shard, synth


def test_balanced_ranges_cover_and_balance():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(3, 0.5, size=1001)
    for world in (1, 2, 3, 8):
        rr = shard.balanced_ranges(costs, world)
        assert rr[0][0] == 0 and rr[-1][1] == len(costs)
        assert all(a[1] == b[0] for a, b in zip(rr, rr[1:]))
        sums = [costs[a:b].sum() for a, b in rr]
        assert max(sums) - min(sums) <= 2 * costs.max()
    assert shard.balanced_ranges([], 2) == [(0, 0), (0, 0)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


RECORD = np.dtype([("ligand_id", np.uint64), ("best_fp64", np.float64, 8),
                   ("best_index", np.int32, 8), ("best_genotype", np.float32, (8, 23))])
SEARCH = dict(pop=32, generations=3, seed=5)


def _setup():
    from oracle import oracle as o
    pk = synth.make_pocket(300, 6.0, seed=3)
    ligs = synth.make_ligands(np.random.Generator(np.random.Philox(8)),
                              np.array([6, 30, 12, 9, 24, 15, 40, 8, 18]),
                              np.array([1, 5, 2, 0, 4, 3, 6, 0, 2]), id_base=70)
    P = o.Params(synth.TYPE_PARAMS)
    pks = o.pocket_from(pk)
    return o, ligs, P, pks, o.grid_build(pks, P, n_threads=1)


def _dock_records(o, ligs, P, pks, grid):
    r = o.dock_batch(ligs, P, pks, grid, SEARCH["pop"], SEARCH["generations"], seed=SEARCH["seed"],
                     n_threads=1)
    out = np.zeros(ligs.n_ligands, RECORD)
    out["ligand_id"] = ligs.ligand_id
    out["best_fp64"] = r["best64"]
    out["best_index"] = r["best_idx"]
    for l in range(ligs.n_ligands):
        out["best_genotype"][l] = r["geno"][l][r["best_idx"][l]]
    return out


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    o, ligs, P, pks, grid = _setup()
    costs = shard.ligand_costs(ligs.atom_off, ligs.tors_off)
    a, b = shard.balanced_ranges(costs, world)[rank]
    mine = _dock_records(o, ligs.subset(np.arange(a, b)), P, pks, grid)
    allrec = shard.gather_records(mine)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((allrec.tobytes(), (a, b), float(t.item())))
    dist.destroy_process_group()


def test_two_rank_gloo_sharded_docking_equals_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    raw, first, tmax = q.get(timeout=300)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    got = np.frombuffer(raw, RECORD)
    o, ligs, P, pks, grid = _setup()
    ref = _dock_records(o, ligs, P, pks, grid)
    assert 0 < first[1] < ligs.n_ligands          # both ranks docked something
    assert got.tobytes() == ref.tobytes()
    np.testing.assert_array_equal(got["ligand_id"], ligs.ligand_id)
    assert tmax == 2.0
