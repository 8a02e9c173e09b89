"""The no-grid and Lamarckian searches at the full c2 size (1,000 ligands x
1,024 poses x 50 generations, graph launch, the launch shape bench.py uses),
checked against the oracle on sampled outputs: GA steps replayed bit-exactly
where the oracle can replay them, FP32 scores of sampled poses within the
per-pose bar (1e-4 relative or 1e-3 absolute; poses within 2e-4 A of a score
discontinuity are counted apart), and the final records."""
import math

import numpy as np
import pytest

from helpers import (MARGIN, OracleSide, PARAMS, branch_ok, gpu_ligands, gpu_pocket, near_ok_grid,
                     pairwise_jumps, within)
from oracle import oracle as o
from paper_2509_12232_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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
def c2(dock):
    pk, ligs, w = synth.make_workload("c2")
    pocket = gpu_pocket(dock, pk)
    gl = gpu_ligands(dock, pocket, ligs)
    return dict(pk=pk, ligs=ligs, w=w, pocket=pocket, gl=gl, side=OracleSide(pk, ligs),
                P=o.Params(PARAMS), pks=o.pocket_from(pk),
                prot=np.stack([pk.x, pk.y, pk.z], 1).astype(np.float64))


def _traced(dock, c2, **kw):
    w, gl = c2["w"], c2["gl"]
    nl, pop, gens = c2["ligs"].n_ligands, w.pop, w.generations
    tot = int(gl.geno_offsets(pop)[-1])
    tg = torch.zeros(gens * tot, dtype=torch.float32, device="cuda")
    ts = torch.zeros(gens * nl * pop, dtype=torch.float32, device="cuda")
    job = dock.dock_batch(c2["pocket"], gl, pop, gens, seed=0, use_graph=1, trace_genotypes=tg,
                          trace_scores=ts, stream=torch.cuda.current_stream(), **SEARCH, **kw)
    res = dock.dock_results(job)
    job.close()
    goff = gl.geno_offsets(pop)

    def geno(l, g):
        G = 7 + c2["ligs"].n_tors(l)
        base = g * tot + int(goff[l])
        return tg[base: base + pop * G].cpu().numpy().reshape(pop, G)

    def scores(l, g):
        return ts[g * nl * pop + l * pop: g * nl * pop + (l + 1) * pop].cpu().numpy()
    return res, geno, scores


def _sample_ligands(c2, n=6, seed=7):
    rng = np.random.default_rng(seed)
    na = np.diff(c2["ligs"].atom_off)
    return sorted(set(rng.choice(c2["ligs"].n_ligands, n, replace=False).tolist() +
                      [int(np.argmax(na))]))


def _pairwise_oracle(c2, l, genos):
    """FP64 pairwise score (inter over every protein atom within 8 A, plus
    intra) and the distance of the pose to a score discontinuity."""
    lig = c2["side"].lig(l)
    score, margin = [], []
    for g in genos:
        xyz = o.pose(lig, g, c2["pk"].center)
        e_intra, m_intra = o.intra(lig, c2["P"], xyz)
        score.append(o.inter_pairwise(lig, c2["P"], c2["pks"], xyz) + e_intra)
        d = np.linalg.norm(xyz[:, None, :] - c2["prot"][None], axis=2)
        margin.append(min(m_intra, float(np.abs(d - 8.0).min())))
    return np.array(score), np.array(margin)


def _near_pairwise(c2, l, genos, got, ref, ok, near, **bar):
    """Margin poses that miss the bar must meet it against a branch value."""
    lig = c2["side"].lig(l)
    for i in np.nonzero(~ok & near)[0]:
        xyz = o.pose(lig, genos[i], c2["pk"].center)
        ok[i] = branch_ok(got[i], ref[i], pairwise_jumps(lig, c2["P"], c2["pks"], xyz), **bar)
    return ok


_near_grid = near_ok_grid


def test_nogrid_c2_full_size_sampled(dock, c2):
    w, ligs = c2["w"], c2["ligs"]
    pop, gens = w.pop, w.generations
    dock.dock_autotune(c2["pocket"], c2["gl"], pop, 4, stream=torch.cuda.current_stream(),
                       inter=dock.DOCK_INTER_PAIRWISE)
    res, geno, scores = _traced(dock, c2, inter=dock.DOCK_INTER_PAIRWISE)
    rng = np.random.default_rng(11)
    checked = near = 0
    for l in _sample_ligands(c2):
        k, lid = ligs.n_tors(l), int(ligs.ligand_id[l])
        for g in (1, 25, gens - 1):
            exp = o.ga_step(k, pop, SEARCH["p_cross"], SEARCH["p_mut"], 0, lid, g,
                            geno(l, g - 1), scores(l, g - 1))
            np.testing.assert_array_equal(geno(l, g).view(np.uint32), exp.view(np.uint32),
                                          err_msg="ligand %d generation %d" % (l, g))
            sel = rng.choice(pop, 24, replace=False)
            ref, margin = _pairwise_oracle(c2, l, geno(l, g)[sel])
            got = scores(l, g)[sel]
            ok = _near_pairwise(c2, l, geno(l, g)[sel], got, ref, within(got, ref), margin < MARGIN)
            assert ok.all(), (l, g, np.nonzero(~ok)[0][:5])
            checked += sel.size
            near += int((margin < MARGIN).sum())
        # the best 8: FP64 pairwise rescores against the oracle's
        G = 7 + k
        ref64, m64 = _pairwise_oracle(c2, l, res[l]["genotype"][:, :G])
        ok64 = np.abs(res[l]["best_fp64"] - ref64) <= 1e-9 * np.maximum(1.0, np.abs(ref64))
        ok64 = _near_pairwise(c2, l, res[l]["genotype"][:, :G], res[l]["best_fp64"], ref64, ok64,
                              m64 < MARGIN, rel=1e-9, abs_=1e-9)
        assert np.all(ok64), (l, res[l]["best_fp64"], ref64)
        fin = scores(l, gens - 1)
        key = [(np.inf if math.isnan(v) else v, i) for i, v in enumerate(fin.tolist())]
        assert res[l]["best_index"].tolist() == [i for _, i in sorted(key)][:8]
    assert checked >= 400 and near <= checked // 10
    assert np.all(res["status"] == 0)
    assert np.all(res["exact_evals"] == pop * gens)


def test_lamarckian_c2_full_size_sampled(dock, c2):
    """With AutoDock's local-search settings (6% of each generation, up to
    300 iterations): every sampled individual's FP32 score, refined or not,
    is the score of its genotype; the best records are the final
    population's; the local search adds evaluations."""
    w, ligs = c2["w"], c2["ligs"]
    pop, gens = w.pop, w.generations
    ls = dock.ls_params(rate=0.06, max_its=300, max_succ=4, max_fail=4, rho=1.0, rho_lb=0.01)
    dock.dock_autotune(c2["pocket"], c2["gl"], pop, 4, stream=torch.cuda.current_stream())
    res, geno, scores = _traced(dock, c2, ls=ls)
    side = c2["side"]
    rng = np.random.default_rng(13)
    checked = near = 0
    for l in _sample_ligands(c2, seed=9):
        for g in (0, 25, gens - 1):
            sel = rng.choice(pop, 32, replace=False)
            ref = side.score(l, geno(l, g)[sel])
            got = scores(l, g)[sel]
            ok = _near_grid(side, l, geno(l, g)[sel], got, ref["score"], within(got, ref["score"]),
                            ref["margin"] < MARGIN)
            assert ok.all(), (l, g, np.nonzero(~ok)[0][:5])
            checked += sel.size
            near += int((ref["margin"] < MARGIN).sum())
        G = 7 + ligs.n_tors(l)
        fin = scores(l, gens - 1)
        key = [(np.inf if math.isnan(v) else v, i) for i, v in enumerate(fin.tolist())]
        order = [i for _, i in sorted(key)][:8]
        assert res[l]["best_index"].tolist() == order
        np.testing.assert_array_equal(res[l]["genotype"][:, :G], geno(l, gens - 1)[order])
        ref = side.score(l, res[l]["genotype"][:, :G])
        ok64 = _near_grid(side, l, res[l]["genotype"][:, :G], res[l]["best_fp64"], ref["score"],
                          within(res[l]["best_fp64"], ref["score"], rel=1e-5, abs_=1e-4),
                          ref["margin"] < MARGIN, rel=1e-5, abs_=1e-4)
        assert np.all(ok64)
    assert checked >= 500 and near <= checked // 20
    assert np.all(res["status"] == 0)
    assert np.all(res["exact_evals"] > pop * gens)


@pytest.mark.parametrize("mode", ["plain", "lga", "nogrid"])
def test_c2_free_running_groups_match_the_joined_schedule(dock, c2, mode):
    """At the full c2 size an untraced search runs each lanes-per-pose group's
    generations on its own stream, joined once (about 30 work items per
    persistent CTA and generation); a score trace makes every generation join.
    The result records of the two schedules are identical field by field."""
    w, gl, nl = c2["w"], c2["gl"], c2["ligs"].n_ligands
    kw = dict(p_cross=0.8, p_mut=0.02)
    if mode == "lga":
        kw["ls"] = dock.ls_params(0.06, 300)
    if mode == "nogrid":
        kw["inter"] = dock.DOCK_INTER_PAIRWISE
    ts = torch.zeros(w.generations * nl * w.pop, dtype=torch.float32, device="cuda")
    out = []
    for trace in (None, ts):
        job = dock.dock_batch(c2["pocket"], gl, w.pop, w.generations, seed=1, use_graph=1,
                              trace_scores=trace, stream=torch.cuda.current_stream(), **kw)
        out.append(dock.dock_results(job))
        job.close()
    free, joined = out
    assert np.all(free["status"] == 0)
    for name in free.dtype.names:
        np.testing.assert_array_equal(free[name], joined[name], err_msg=name)
