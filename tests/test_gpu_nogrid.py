"""The no-grid search (dock_batch with inter = DOCK_INTER_PAIRWISE) against the
oracle: the GA replayed on the CPU from the GPU's own FP32 scores must give
bit-identical populations every generation; every FP32 score must match the
oracle's pairwise score (inter over every protein atom within 8 A, plus
intra) within 1e-4 relative or 1e-3 absolute; the best 8 rescored in FP64 on
the GPU must match the oracle's FP64 pairwise score to 1e-9 relative. Poses
with a pair within 2e-4 A of the 8 A cutoff are counted apart."""
import math

import numpy as np
import pytest

from helpers import MARGIN, PARAMS, branch_ok, gpu_ligands, pairwise_jumps, within
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
def setup(dock):
    pk, _, _ = synth.make_workload("c1")
    rng = np.random.Generator(np.random.Philox(77))
    ligs = synth.make_ligands(rng, np.array([9, 26, 44, 70]), np.array([1, 4, 7, 12]), id_base=900)
    pocket = dock.dock_create_pocket(pk.x, pk.y, pk.z, pk.q, pk.type, pk.center, pk.radius,
                                     pk.spacing, PARAMS)
    gl = gpu_ligands(dock, pocket, ligs)
    return dict(pk=pk, ligs=ligs, pocket=pocket, gl=gl, P=o.Params(PARAMS), pks=o.pocket_from(pk),
                prot=np.stack([pk.x, pk.y, pk.z], 1).astype(np.float64))


def _oracle(setup, l, genos):
    lig = o.Ligand(**setup["ligs"].ligand(l))
    score, margin = [], []
    for g in genos:
        xyz = o.pose(lig, g, setup["pk"].center)
        e_intra, m_intra = o.intra(lig, setup["P"], xyz)
        score.append(o.inter_pairwise(lig, setup["P"], setup["pks"], xyz) + e_intra)
        d = np.linalg.norm(xyz[:, None, :] - setup["prot"][None], axis=2)
        margin.append(min(m_intra, float(np.abs(d - 8.0).min())))
    return np.array(score), np.array(margin)


def _check_near(setup, l, genos, got, ref, ok, near, **bar):
    """Poses within the margin of the cutoff that miss the bar must meet it
    against one of their branch values."""
    lig = o.Ligand(**setup["ligs"].ligand(l))
    for i in np.nonzero(~ok & near)[0]:
        xyz = o.pose(lig, genos[i], setup["pk"].center)
        ok[i] = branch_ok(got[i], ref[i], pairwise_jumps(lig, setup["P"], setup["pks"], xyz), **bar)
    return ok


@pytest.mark.parametrize("lanes", [0, 8, 2, "tuned"])
def test_nogrid_search_replay(dock, setup, lanes):
    """lanes 0: lanes per pose picked by ligand size (several launch groups);
    8 and 2: every ligand forced to that many lanes per pose; tuned: the
    launch shape dock_autotune picks for the no-grid search."""
    ligs, gl, pocket = setup["ligs"], setup["gl"], setup["pocket"]
    nl, pop, gens, seed = ligs.n_ligands, 48, 4, 3
    if lanes == "tuned":
        tune = dock.dock_autotune(pocket, gl, pop, 2, stream=torch.cuda.current_stream(),
                                  inter=dock.DOCK_INTER_PAIRWISE)
        assert len(tune["table"]) >= 2 and 0 <= tune["best"] < len(tune["table"])
        lanes = 0
    goff = gl.geno_offsets(pop)
    tot = int(goff[-1])
    tg = torch.zeros(gens * tot, dtype=torch.float32, device="cuda")
    ts = torch.zeros(gens * nl * pop, dtype=torch.float32, device="cuda")
    job = dock.dock_batch(pocket, gl, pop, gens, seed=seed, trace_genotypes=tg, trace_scores=ts,
                          stream=torch.cuda.current_stream(), inter=dock.DOCK_INTER_PAIRWISE,
                          lanes_per_pose=lanes, **SEARCH)
    res = dock.dock_results(job)
    tg, ts = tg.cpu().numpy(), ts.cpu().numpy()
    R = setup["pk"].radius
    near_total = checked = 0
    for l in range(nl):
        k = ligs.n_tors(l)
        G = 7 + k
        lid = int(ligs.ligand_id[l])

        def geno(g):
            base = g * tot + int(goff[l])
            return tg[base: base + pop * G].reshape(pop, G)

        def scores(g):
            return ts[g * nl * pop + l * pop: g * nl * pop + (l + 1) * pop]
        for g in range(gens):
            exp = o.ga_init(k, pop, R, seed, lid) if g == 0 else \
                o.ga_step(k, pop, SEARCH["p_cross"], SEARCH["p_mut"], seed, lid, g, geno(g - 1),
                          scores(g - 1))
            np.testing.assert_array_equal(geno(g).view(np.uint32), exp.view(np.uint32),
                                          err_msg="ligand %d generation %d" % (l, g))
            ref, margin = _oracle(setup, l, geno(g))
            near = margin < MARGIN
            ok = _check_near(setup, l, geno(g), scores(g), ref, within(scores(g), ref), near)
            bad = np.nonzero(~ok)[0]
            assert bad.size == 0, (l, g, bad[:5], scores(g)[bad[:5]], ref[bad[:5]])
            near_total += int(near.sum())
            checked += pop
        r = res[l]
        fin = scores(gens - 1)
        key = [(np.inf if math.isnan(v) else v, i) for i, v in enumerate(fin.tolist())]
        order = [i for _, i in sorted(key)][:8]
        assert r["best_index"].tolist() == order
        ref64, margin64 = _oracle(setup, l, geno(gens - 1)[order])
        ok64 = np.abs(r["best_fp64"] - ref64) <= 1e-9 * np.maximum(1.0, np.abs(ref64))
        ok64 = _check_near(setup, l, geno(gens - 1)[order], r["best_fp64"], ref64, ok64,
                           margin64 < MARGIN, rel=1e-9, abs_=1e-9)
        assert np.all(ok64), (l, r["best_fp64"], ref64)
        assert int(r["exact_evals"]) == pop * gens
    # a pose of the 70-atom ligand has ~2,000 intra pairs and often protein atoms
    # near 8 A: a pair within the margin occurs in a few percent of the poses
    assert near_total <= 0.15 * checked
    job.close()


def test_nogrid_search_is_invariant_under_joint_rigid_motion(dock, setup):
    """Protein and pocket centre moved together: the generation-0 population
    (drawn relative to the centre) scores the same within rounding, pose by
    pose, except where a pair sits at the 8 A cutoff (the moved coordinates
    round differently)."""
    pk, ligs = setup["pk"], setup["ligs"]
    s = np.array([4.0, -8.0, 2.0], np.float32)
    pocket2 = dock.dock_create_pocket(pk.x + s[0], pk.y + s[1], pk.z + s[2], pk.q, pk.type,
                                      np.asarray(pk.center, np.float32) + s, pk.radius, pk.spacing,
                                      PARAMS)
    gl2 = gpu_ligands(dock, pocket2, ligs)
    pop = 256
    out = []
    for pocket, gl in ((setup["pocket"], setup["gl"]), (pocket2, gl2)):
        ts = torch.zeros(ligs.n_ligands * pop, dtype=torch.float32, device="cuda")
        job = dock.dock_batch(pocket, gl, pop, 1, seed=8, stream=torch.cuda.current_stream(),
                              trace_scores=ts, inter=dock.DOCK_INTER_PAIRWISE, **SEARCH)
        dock.dock_results(job)
        out.append(ts.cpu().numpy())
        job.close()
    ok = within(out[1], out[0])
    assert ok.mean() >= 0.98, (ok.mean(), np.nonzero(~ok)[0][:5])


def test_nogrid_invalid_settings(dock, setup):
    pocket, gl = setup["pocket"], setup["gl"]
    with pytest.raises(dock.DockError):
        dock.dock_batch(pocket, gl, 16, 2, inter=2)
    with pytest.raises(dock.DockError):
        dock.dock_batch(pocket, gl, 16, 2, inter=dock.DOCK_INTER_PAIRWISE, lanes_per_pose=3)
    with pytest.raises(dock.DockError):
        dock.dock_batch(pocket, gl, 16, 2, inter=dock.DOCK_INTER_PAIRWISE,
                        ls=dock.ls_params(rate=0.1))
