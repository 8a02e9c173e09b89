"""Solis-Wets local search on the GPU against the oracle's, through the C ABI.

Each GPU chain is replayed by the oracle's Solis-Wets fed the GPU's own probe
scores (recorded in the trace): the refined genotype and score must then be
bit-identical (the probe arithmetic is correctly rounded FP32 on both sides),
and every probe score the GPU computed must lie within the per-pose bar of the
oracle's FP64 score of the oracle's own probe (1e-4 relative or 1e-3
absolute; probes within 2e-4 A of a score discontinuity are counted apart).
The Lamarckian search (dock_batch with ls) is replayed generation by
generation: the GA step from the GPU's traced population, the selection draw,
then each selected individual's chain."""
import math

import numpy as np
import pytest

from helpers import MARGIN, OracleSide, branch_jumps, branch_ok, gpu_ligands, gpu_pocket, within
from oracle import oracle as o
from paper_2509_12232_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import to_dev  # noqa: E402

SEARCH = dict(p_cross=0.8, p_mut=0.02)


@pytest.fixture(scope="module")
def dock():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2509_12232_gb300 import build
    build.build()
    from paper_2509_12232_gb300 import dock as d
    d.lib()
    return d


@pytest.fixture(scope="module")
def setup(dock):
    pk, _, _ = synth.make_workload("c1")
    rng = np.random.Generator(np.random.Philox(4242))
    # sizes for 1, 2, 4 and 8 lanes per pose at 16 atoms per lane, plus a tiny one
    ligs = synth.make_ligands(rng, np.array([12, 25, 50, 90, 3]), np.array([2, 5, 9, 16, 0]),
                              id_base=800)
    side = OracleSide(pk, ligs)
    pocket = gpu_pocket(dock, pk)
    gl = gpu_ligands(dock, pocket, ligs)
    return dict(pk=pk, ligs=ligs, side=side, pocket=pocket, gl=gl)


class Probes:
    """GPU probe scores next to the oracle's FP64 scores of the same probes."""

    def __init__(self):
        self.gpu, self.ref, self.margin, self.src = [], [], [], []

    def add(self, gpu, ref, side, l, geno):
        self.gpu.append(float(gpu))
        self.ref.append(float(ref["score"][0]))
        self.margin.append(float(ref["margin"][0]))
        self.src.append((side, l, np.array(geno)))

    def check(self, what):
        g, r, m = (np.array(v, np.float64) for v in (self.gpu, self.ref, self.margin))
        near = m < MARGIN
        ok = within(g, r)
        for i in np.nonzero(~ok & near)[0]:
            side, l, geno = self.src[i]
            ok[i] = branch_ok(g[i], r[i], branch_jumps(side, l, geno))
        bad = np.nonzero(~ok)[0]
        assert bad.size == 0, (what, bad[:5], g[bad[:5]], r[bad[:5]])
        # a 90-atom ligand has ~4,000 intra pairs: one of them lies within the
        # margin of the 8 A cutoff in several percent of its poses
        assert near.mean() <= 0.1, (what, int(near.sum()), len(g))
        return len(g)


def _replay_chain(side, l, k, ls_o, seed, lig_id, gen, ind, x0, row, probes):
    """The oracle's chain from x0 with the GPU's recorded probe scores."""
    f0 = float(row[0])

    def obj(g, it, which):
        v = float(row[2 + 2 * it + which])
        ref = side.score(l, g[None])
        probes.add(v, ref, side, l, g)
        return v
    return o.solis_wets(k, ls_o, seed, lig_id, gen, ind, x0, f0, obj)


@pytest.mark.parametrize("max_its", [1, 40])
def test_standalone_chains_replay_bit_exact(dock, setup, max_its):
    ligs, side = setup["ligs"], setup["side"]
    R = setup["pk"].radius
    seed, gen = 21, 7
    pl, genos = [], []
    for l in range(ligs.n_ligands):
        k = ligs.n_tors(l)
        g = o.ga_init(k, 9, R, 100 + l, int(ligs.ligand_id[l]))
        g[:3, :3] *= 1.8  # some start inside the protein shell
        for row in g:
            pl.append(l)
            genos.append(np.r_[row, np.zeros(23 - 7 - k, np.float32)])
    pl = np.array(pl, np.int32)
    genos = np.array(genos, np.float32)
    n = len(pl)
    ls = dock.ls_params(max_its=max_its)
    ls_o = o.LsParams(max_its=max_its)
    dg = to_dev(torch, genos)
    sc = torch.zeros(n, dtype=torch.float32, device="cuda")
    tr = torch.full((n, 2 + 2 * max_its), float("nan"), dtype=torch.float32, device="cuda")
    ev = torch.zeros(n, dtype=torch.int32, device="cuda")
    dock.dock_local_search(setup["pocket"], setup["gl"], ls, seed, gen, to_dev(torch, pl), dg, sc,
                           trace=tr, evals=ev)
    torch.cuda.synchronize()
    out, sc, tr, ev = dg.cpu().numpy(), sc.cpu().numpy(), tr.cpu().numpy(), ev.cpu().numpy()
    probes, starts = Probes(), Probes()
    improved = 0
    for p in range(n):
        l = int(pl[p])
        k = ligs.n_tors(l)
        G = 7 + k
        ref0 = side.score(l, genos[p, :G][None])
        starts.add(tr[p, 0], ref0, side, l, genos[p, :G])
        x, f, its, nev = _replay_chain(side, l, k, ls_o, seed, int(ligs.ligand_id[l]), gen, p,
                                       genos[p, :G], tr[p], probes)
        np.testing.assert_array_equal(out[p, :G].view(np.uint32), x.view(np.uint32),
                                      err_msg="pose %d" % p)
        np.testing.assert_array_equal(out[p, G:], genos[p, G:])  # genes beyond G untouched
        assert np.float32(f).view(np.uint32) == sc[p].view(np.uint32), (p, f, sc[p])
        assert its == int(tr[p, 1]) and nev == int(ev[p])
        improved += f < tr[p, 0]
    starts.check("start scores")
    assert probes.check("probes") >= n
    if max_its > 1:
        assert improved >= n // 2


def test_lamarckian_search_replay(dock, setup):
    ligs, side, gl, pocket = setup["ligs"], setup["side"], setup["gl"], setup["pocket"]
    nl = ligs.n_ligands
    pop, gens, seed, rate, max_its = 40, 4, 5, 0.3, 30
    goff = gl.geno_offsets(pop)
    tot = int(goff[-1])
    w = 2 + 2 * max_its
    tg = torch.zeros(gens * tot, dtype=torch.float32, device="cuda")
    ts = torch.zeros(gens * nl * pop, dtype=torch.float32, device="cuda")
    tl = torch.full((gens * nl * pop * w,), float("nan"), dtype=torch.float32, device="cuda")
    job = dock.dock_batch(pocket, gl, pop, gens, seed=seed, trace_genotypes=tg, trace_scores=ts,
                          stream=torch.cuda.current_stream(), ls=dock.ls_params(rate, max_its),
                          trace_ls=tl, **SEARCH)
    res = dock.dock_results(job)
    tg, ts = tg.cpu().numpy(), ts.cpu().numpy()
    tl = tl.cpu().numpy().reshape(gens, nl, pop, w)
    ls_o = o.LsParams(rate=rate, max_its=max_its)
    R = setup["pk"].radius
    probes, plain = Probes(), Probes()
    chains = 0
    for l in range(nl):
        k = ligs.n_tors(l)
        G = 7 + k
        lid = int(ligs.ligand_id[l])

        def geno(g):
            base = g * tot + int(goff[l])
            return tg[base: base + pop * G].reshape(pop, G)

        def scores(g):
            return ts[g * nl * pop + l * pop: g * nl * pop + (l + 1) * pop]
        evals = pop * gens
        for g in range(gens):
            pre = o.ga_init(k, pop, R, seed, lid) if g == 0 else \
                o.ga_step(k, pop, SEARCH["p_cross"], SEARCH["p_mut"], seed, lid, g, geno(g - 1),
                          scores(g - 1))
            cur, cs = geno(g), scores(g)
            for i in range(pop):
                if not o.ls_selected(rate, seed, lid, g, i):
                    np.testing.assert_array_equal(cur[i].view(np.uint32), pre[i].view(np.uint32),
                                                  err_msg="l %d g %d i %d" % (l, g, i))
                    ref = side.score(l, cur[i][None])
                    plain.add(cs[i], ref, side, l, cur[i])
                    continue
                row = tl[g, l, i]
                ref = side.score(l, pre[i][None])  # the chain starts from the scored child
                plain.add(row[0], ref, side, l, pre[i])
                x, f, its, nev = _replay_chain(side, l, k, ls_o, seed, lid, g, i, pre[i], row, probes)
                np.testing.assert_array_equal(cur[i].view(np.uint32), x.view(np.uint32),
                                              err_msg="chain l %d g %d i %d" % (l, g, i))
                assert np.float32(f).view(np.uint32) == cs[i].view(np.uint32)
                assert its == int(row[1])
                evals += nev
                chains += 1
        # results: best 8 of the final (refined) population, evaluations counted
        r = res[l]
        fin = scores(gens - 1)
        key = [(np.inf if math.isnan(v) else v, i) for i, v in enumerate(fin.tolist())]
        order = [i for _, i in sorted(key)][:8]
        assert r["best_index"].tolist() == order
        assert int(r["exact_evals"]) == evals
    plain.check("scores")
    probes.check("probes")
    assert chains >= 0.2 * nl * pop * gens
    job.close()


def test_lamarckian_improves_on_the_plain_ga(dock, setup):
    pocket, gl, nl = setup["pocket"], setup["gl"], setup["ligs"].n_ligands
    best = {}
    for name, ls in (("plain", None), ("lga", dock.ls_params(0.06, 300))):
        job = dock.dock_batch(pocket, gl, 64, 8, seed=2, stream=torch.cuda.current_stream(), ls=ls)
        best[name] = dock.dock_results(job)["best_fp64"][:, 0].copy()
        job.close()
    assert np.all(best["lga"] <= best["plain"] + 1e-6)
    assert np.mean(best["plain"] - best["lga"]) > 0.5


@pytest.mark.parametrize("mode", ["plain", "lga", "pairwise"])
def test_free_running_groups_match_the_joined_schedule(dock, setup, mode):
    """Untraced, each lanes-per-pose group (here four: 1, 2, 4 and 8 lanes) runs
    all its generations on its own stream and the streams join once; with a
    score trace every generation joins. A ligand's arithmetic does not depend
    on the schedule, so the result records are identical field by field."""
    pocket, gl, nl = setup["pocket"], setup["gl"], setup["ligs"].n_ligands
    pop, gens = 64, 8
    ls = dock.ls_params(0.06, 300) if mode == "lga" else None
    inter = dock.DOCK_INTER_PAIRWISE if mode == "pairwise" else dock.DOCK_INTER_GRID
    ts = torch.zeros(gens * nl * pop, dtype=torch.float32, device="cuda")
    out = []
    for trace in (None, ts):
        job = dock.dock_batch(pocket, gl, pop, gens, seed=3, stream=torch.cuda.current_stream(),
                              ls=ls, inter=inter, trace_scores=trace, **SEARCH)
        out.append(dock.dock_results(job))
        job.close()
    free, joined = out
    assert np.all(free["status"] == 0)
    for name in free.dtype.names:
        np.testing.assert_array_equal(free[name], joined[name], err_msg=name)


def test_bad_pose_ligand_and_invalid_settings(dock, setup):
    pocket, gl = setup["pocket"], setup["gl"]
    g = np.zeros((3, 23), np.float32)
    g[:, 3] = 1.0
    dg = to_dev(torch, g)
    sc = torch.zeros(3, dtype=torch.float32, device="cuda")
    pl = to_dev(torch, np.array([0, 7, -2], np.int32))
    dock.dock_local_search(pocket, gl, dock.ls_params(max_its=5), 1, 0, pl, dg, sc)
    torch.cuda.synchronize()
    s = sc.cpu().numpy()
    assert np.isfinite(s[0]) and np.isnan(s[1]) and np.isnan(s[2])
    np.testing.assert_array_equal(dg.cpu().numpy()[1:], g[1:])
    for bad in (dict(max_its=0), dict(max_its=10 ** 6), dict(max_succ=0), dict(rho=0.0),
                dict(rho=float("inf")), dict(rho_lb=float("nan"))):
        with pytest.raises(dock.DockError) as e:
            dock.dock_local_search(pocket, gl, dock.ls_params(**bad), 1, 0, pl, dg, sc)
        assert e.value.status == dock.DOCK_EINVAL
    with pytest.raises(dock.DockError):
        dock.dock_batch(pocket, gl, 16, 2, ls=dock.ls_params(rate=1.5))
    with pytest.raises(dock.DockError):
        dock.dock_batch(pocket, gl, 16, 2, ls=dock.ls_params(rate=0.1, max_its=0))
    # an empty call is a no-op
    dock.dock_local_search(pocket, gl, dock.ls_params(), 1, 0, pl[:0], dg[:0], sc[:0])
