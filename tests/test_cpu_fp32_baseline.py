"""The FP32 auto-vectorised CPU baseline (oracle/simd_fp32.c, the paper's
own style of hot path: FP32 SoA loops under #pragma omp simd). It is a
second CPU reference point for the benchmark; these tests check that it
computes the same method: its FP32 scores against the FP64 oracle within the
per-pose bar (poses near a discontinuity against their branch values), and
its search genotypes against the oracle's GA replayed on its own scores."""
import numpy as np
import pytest

from helpers import MARGIN, OracleSide, branch_jumps, branch_ok, within
from oracle import oracle as o
from paper_2509_12232_gb300 import synth


@pytest.fixture(scope="module")
def side():
    pk = synth.make_pocket(600, 8.0, seed=5)
    rng = np.random.Generator(np.random.Philox(31))
    ligs = synth.make_ligands(rng, np.array([24, 9, 40]), np.array([4, 1, 7]), id_base=40)
    return OracleSide(pk, ligs)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_fp32_scores_match_the_fp64_oracle(side, l):
    lig = side.lig(l)
    g = o.ga_init(lig.k, 400, side.pk.radius, 3 + l, 55)
    g[:150, :3] *= 1.6                       # some poses against the protein wall
    ref = side.score(l, g)
    got = o.cpu32_score_poses(lig, side.P, side.grid, side.pk.center, g).astype(np.float64)
    ok = within(got, ref["score"])
    for i in np.nonzero(~ok & (ref["margin"] < MARGIN))[0]:
        ok[i] = branch_ok(got[i], ref["score"][i], branch_jumps(side, l, g[i]))
    assert np.all(ok), (np.nonzero(~ok)[0][:5], got[~ok][:5], ref["score"][~ok][:5])
    assert np.ptp(ref["score"]) > 1.0        # not a constant


def test_fp32_search_genotypes_are_the_oracle_ga_on_its_scores(side):
    pop, gens, seed = 96, 4, 9
    sub = side.ligs.subset([0])
    r = o.cpu32_dock_batch(sub, side.P, side.pks, side.grid, pop, gens, seed=seed, n_threads=1,
                           trace=True)
    k = sub.n_tors(0)
    lid = int(sub.ligand_id[0])
    tg, ts = r["trace_geno"], r["trace_score"]
    np.testing.assert_array_equal(tg[0], o.ga_init(k, pop, side.pk.radius, seed, lid))
    for g in range(1, gens):
        exp = o.ga_step(k, pop, 0.8, 0.02, seed, lid, g, tg[g - 1], ts[g - 1])
        np.testing.assert_array_equal(tg[g].view(np.uint32), exp.view(np.uint32))
    # the scores it traced are its own FP32 scores of those genotypes
    lig = side.lig(0)
    np.testing.assert_array_equal(ts[-1], o.cpu32_score_poses(lig, side.P, side.grid, side.pk.center,
                                                              tg[-1]))
    np.testing.assert_array_equal(r["score"][0], ts[-1])
    assert r["best"][0] == int(np.argmin(ts[-1]))


def test_fp32_batch_threads_do_not_change_results(side):
    a = o.cpu32_dock_batch(side.ligs, side.P, side.pks, side.grid, 64, 3, seed=2, n_threads=1)
    b = o.cpu32_dock_batch(side.ligs, side.P, side.pks, side.grid, 64, 3, seed=2, n_threads=3)
    np.testing.assert_array_equal(a["score"], b["score"])
