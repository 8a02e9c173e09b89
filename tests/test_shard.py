"""Multi-process sharding of ligands (gloo, world size 2, CPU): the ranks'
contiguous ranges cover the batch exactly once and balance the cost; each
rank's per-ligand results (here: a deterministic stand-in per ligand id) are
gathered on rank 0 unchanged; the step time is the maximum over ranks."""
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


def _worker(rank, world, port, atom_off, tors_off, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = shard.ligand_costs(atom_off, tors_off)
    a, b = shard.balanced_ranges(costs, world)[rank]
    mine = torch.arange(a, b, dtype=torch.int64)
    # per-ligand "result": a deterministic function of the ligand index
    res = (mine * 2654435761) % 1000003
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([b - a]))
    m = int(max(s.item() for s in sizes))
    pad = torch.full((m,), -1, dtype=torch.int64)
    pad[:b - a] = res
    got = [torch.zeros(m, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(got, pad)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        allres = torch.cat([g[:int(s.item())] for g, s in zip(got, sizes)])
        out.put((allres.numpy().tolist(), float(t.item())))
    dist.destroy_process_group()


def test_two_rank_gloo_sharding():
    ligs = synth.make_ligands(np.random.default_rng(1), np.full(37, 20) + np.arange(37), np.zeros(37, int))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ligs.atom_off, ligs.tors_off, q))
             for r in range(2)]
    for p in procs:
        p.start()
    res, tmax = q.get(timeout=120)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert res == [(i * 2654435761) % 1000003 for i in range(37)]
    assert tmax == 2.0
