"""Pins of the oracle's Solis-Wets local search (the Lamarckian variant of the
GA: AutoDock's search as Morris et al. 1998 describe it, the random search
with bias of Solis & Wets 1981). Each pin is a property of the method that
does not restate the oracle's code: the closed-form length of a search that
never succeeds, the symmetry of the two probes about the current point, the
step size schedule (rho halves after four failures, doubles after four
successes) seen in the probes, the bias following successful directions,
convergence on a convex bowl, monotone improvement on docking scores, and the
selection rate."""
import math

import numpy as np
import pytest

from oracle import oracle as o
from paper_2509_12232_gb300 import synth

X0 = np.array([0.5, -0.25, 1.0, 1.0, 0.0, 0.0, 0.0], np.float32)


def _run(k, ls, x0, f0, objective, seed=7, lig=11, gen=3, ind=5):
    calls = []

    def obj(g, it, which):
        v = objective(g, it, which)
        calls.append((it, which, g.copy(), v))
        return v
    x, f, its, ev = o.solis_wets(k, ls, seed, lig, gen, ind, x0, f0, obj)
    return x, f, its, ev, calls


def test_no_success_stops_after_the_contraction_schedule():
    # rho: 1 -> 1/2 -> ... every max_fail failures; the search stops once rho < rho_lb:
    # ceil(log2(rho / rho_lb)) contractions of max_fail iterations, two probes each
    ls = o.LsParams(rho=1.0, rho_lb=0.01, max_fail=4, max_succ=4, max_its=300)
    x, f, its, ev, calls = _run(0, ls, X0, 2.0, lambda g, it, w: 2.0)
    n_con = math.ceil(math.log2(1.0 / 0.01))
    assert its == 4 * n_con and ev == 2 * its
    assert np.array_equal(x, X0) and f == 2.0
    # a probe that only ties is no success either
    ls3 = o.LsParams(rho=0.5, rho_lb=0.1, max_fail=3)
    x, f, its, ev, _ = _run(2, ls3, np.r_[X0, [0.3, -0.2]].astype(np.float32), 1.0,
                            lambda g, it, w: 1.0)
    assert its == 3 * math.ceil(math.log2(0.5 / 0.1)) and ev == 2 * its


def test_max_iterations_bound():
    ls = o.LsParams(max_its=37)
    _, _, its, ev, calls = _run(0, ls, X0, 0.0, lambda g, it, w: float(g[0]))
    assert its == 37 and ev == len(calls) and 37 <= ev <= 74


def test_probes_are_symmetric_about_the_current_point():
    # when the forward probe x + xi fails, the backward probe is x - xi
    k = 3
    x0 = np.r_[X0, [0.4, -1.0, 2.0]].astype(np.float32)
    rng = np.random.default_rng(1)
    w = rng.normal(size=3)
    obj = lambda g, it, which: float(np.float32(np.dot(w, g[:3]) ** 2))  # noqa: E731
    x, f, its, ev, calls = _run(k, o.LsParams(), x0, obj(x0, 0, 0), obj)
    cur = x0.astype(np.float64)
    fcur = obj(x0, 0, 0)
    checked = 0
    for a, b in zip(calls, calls[1:]):
        if a[1] == 0 and b[1] == 1 and a[0] == b[0]:
            # translation genes: fwd + bwd = 2 x (FP32 rounding of the two sums)
            assert np.allclose(a[2][:3] + b[2][:3], 2 * cur[:3], atol=1e-5 * (1 + np.abs(cur[:3]).max()))
            checked += 1
        if a[3] < fcur:
            cur, fcur = a[2].astype(np.float64), a[3]
    last = calls[-1]
    if last[3] < fcur:
        cur, fcur = last[2].astype(np.float64), last[3]
    assert checked > 10
    assert np.array_equal(cur.astype(np.float32), x) and fcur == f


@pytest.mark.parametrize("k", [0, 4])
def test_step_size_schedule_seen_in_the_probes(k):
    # a never-improving objective keeps the bias at zero, so a probe's
    # displacement of gene e is rho sigma_e z with z ~ N(0, 1): translation
    # sigma 1 A, torsion sigma 0.5 rad; rho halves every 4 iterations
    x0 = np.r_[X0, np.zeros(k)].astype(np.float32)
    ls = o.LsParams(rho=1.0, rho_lb=1e-4)
    ratios = {}
    for ind in range(40):
        _, _, its, _, calls = _run(k, ls, x0, 0.0, lambda g, it, w: 1.0, ind=ind)
        for it, which, g, _ in calls:
            if which != 0:
                continue
            d = (g.astype(np.float64) - x0)
            r = list(d[:3] / 1.0) + list(d[7:] / 0.5)
            # torsions wrap: use only displacements well inside (-pi, pi)
            r = [v for j, v in enumerate(r) if j < 3 or abs(d[7 + j - 3]) < 2.5]
            ratios.setdefault(it // 4, []).extend(r)
    for blk, r in ratios.items():
        rms = float(np.sqrt(np.mean(np.square(r))))
        assert 0.8 < rms / 2.0 ** -blk < 1.25, (blk, rms)


def test_step_size_expands_after_successes():
    # every forward probe succeeds (strictly decreasing objective): rho doubles
    # every 4 iterations, and the displacement grows by 2 per 4 iterations
    x0 = X0.copy()
    growth = []
    for ind in range(30):
        cnt = [0]

        def obj(g, it, w):
            cnt[0] += 1
            return -float(cnt[0])
        _, _, its, ev, calls = _run(0, o.LsParams(max_its=24), x0, 0.0, obj, ind=ind)
        assert its == 24 and ev == 24 and all(c[1] == 0 for c in calls)
        prev = x0.astype(np.float64)
        mags = []
        for it, which, g, _ in calls:
            mags.append(np.sqrt(np.mean((g[:3].astype(np.float64) - prev[:3]) ** 2)))
            prev = g.astype(np.float64)
        m = np.array(mags).reshape(6, 4).mean(axis=1)
        growth.append(np.log2(m[5] / m[1]) / 4.0)  # doublings per block of 4
    assert 0.8 < float(np.median(growth)) < 1.2


def test_bias_follows_successful_directions():
    # on a linear objective an unbiased symmetric probe succeeds forward half
    # the time; the bias (0.2 b + 0.4 xi after a forward success) makes the
    # next forward probe point downhill more often
    frac = []
    for seed in range(20):
        _, _, its, _, calls = _run(0, o.LsParams(max_its=100), X0, float(X0[0]),
                                   lambda g, it, w: float(g[0]), seed=seed)
        frac.append(1.0 - sum(c[1] for c in calls) / its)
    assert np.mean(frac) > 0.6


def test_converges_on_a_convex_bowl():
    c = np.array([0.3, -0.2, 0.1])

    def quad(g, it=0, w=0):
        return float(np.sum((g[:3].astype(np.float64) - c) ** 2))
    for seed in range(10):
        x, f, its, ev, _ = _run(0, o.LsParams(), X0, quad(X0), quad, seed=seed)
        assert f < 1e-3 and quad(x) == pytest.approx(f, rel=1e-6)


def test_nan_scores_count_as_infinite():
    # a NaN start is beaten by the first finite probe; NaN probes never win
    x, f, its, ev, calls = _run(0, o.LsParams(max_its=5), X0, float("nan"),
                                lambda g, it, w: 3.0)
    assert f == 3.0 and not np.array_equal(x, X0)
    x, f, its, ev, calls = _run(0, o.LsParams(max_its=5), X0, 3.0,
                                lambda g, it, w: float("nan"))
    assert f == 3.0 and np.array_equal(x, X0)


def test_refinement_lowers_docking_scores():
    pk, _, _ = synth.make_workload("c1")
    rng = np.random.Generator(np.random.Philox(99))
    ligs = synth.make_ligands(rng, np.array([18, 30]), np.array([3, 6]), id_base=70)
    P = o.Params(synth.TYPE_PARAMS)
    grid = o.grid_build(o.pocket_from(pk), P)
    for l in range(2):
        lig = o.Ligand(**ligs.ligand(l))
        k = lig.k
        g0 = o.ga_init(k, 6, pk.radius, 5, int(ligs.ligand_id[l]))
        s0 = o.score_poses(lig, P, grid, pk.center, g0)["score"].astype(np.float32)

        def obj(g, it, w):
            return np.float32(o.score_poses(lig, P, grid, pk.center, g[None])["score"][0])
        gains = []
        for i in range(6):
            x, f, its, ev = o.solis_wets(k, o.LsParams(max_its=60), 5, int(ligs.ligand_id[l]), 0, i,
                                         g0[i], float(s0[i]), obj)
            assert f <= s0[i]
            assert obj(x, 0, 0) == np.float32(f)  # the reported score is the genotype's
            q = x[3:7].astype(np.float64)
            assert abs(np.linalg.norm(q) - 1) < 1e-6
            gains.append(float(s0[i]) - f)
        assert np.mean(gains) > 0


def test_selection_rate_and_stream_separation():
    rate = 0.06
    n = 20000
    sel = np.array([o.ls_selected(rate, 3, 17, g, i) for g in range(4) for i in range(n // 4)])
    assert abs(sel.mean() - rate) < 5 * math.sqrt(rate * (1 - rate) / n)
    assert not any(o.ls_selected(0.0, 3, 17, 1, i) for i in range(200))
    assert all(o.ls_selected(1.0, 3, 17, 1, i) for i in range(200))
    # the local search draws its normals from counters the GA never uses
    for s in (0, 4, 10):
        assert o.normal(3, 17, 2, 5, s) != o.normal(3, 17, 2 | (1 << 31), 5, s)


def test_lamarckian_search_beats_the_plain_ga():
    pk, _, _ = synth.make_workload("c1")
    rng = np.random.Generator(np.random.Philox(5))
    ligs = synth.make_ligands(rng, np.array([14, 22, 30]), np.array([2, 4, 5]), id_base=300)
    P = o.Params(synth.TYPE_PARAMS)
    pks = o.pocket_from(pk)
    grid = o.grid_build(pks, P)
    plain = o.dock_batch(ligs, P, pks, grid, pop=24, generations=6, seed=9)
    lga = o.dock_batch(ligs, P, pks, grid, pop=24, generations=6, seed=9,
                       ls=o.LsParams(rate=0.25, max_its=40))
    assert np.all(lga["best64"][:, 0] <= plain["best64"][:, 0] + 1e-9)
    assert np.mean(plain["best64"][:, 0] - lga["best64"][:, 0]) > 0.1


@pytest.mark.parametrize("direction", ["forward", "backward"])
def test_bias_recursion_autocorrelation(direction):
    # At a fixed rho (no expansion) with every iteration a success in one
    # direction, the accepted displacement a_t = +-(b_t + d_t), d_t iid N(0, s^2).
    # Forward: b' = 0.2 b + 0.4 (b + d) = 0.6 b + 0.4 d  ->  Var b = 0.16/0.64 s^2,
    #   corr(a_t, a_t+1) = (0.6 Var b + 0.4 s^2) / (Var b + s^2) = 0.44.
    # Backward: b' = b - 0.4 (b + d) = 0.6 b - 0.4 d  ->  same Var b,
    #   corr = (0.6 Var b - 0.4 s^2) / (Var b + s^2) = -0.2.
    ls = o.LsParams(max_its=200, max_succ=10 ** 6, max_fail=10 ** 6)
    pairs = []
    for ind in range(30):
        cnt = [0]

        def obj(g, it, w):
            if direction == "backward" and w == 0:
                return 1e30
            cnt[0] += 1
            return -float(cnt[0])
        _, _, its, _, calls = _run(0, ls, X0, 0.0, obj, ind=ind)
        acc = [c[2][:3].astype(np.float64) for c in calls if c[3] < 1e29]
        disp = np.diff(np.array([X0[:3].astype(np.float64)] + acc), axis=0)[20:]
        pairs.append(np.stack([disp[:-1], disp[1:]], 0).reshape(2, -1))
    a = np.concatenate(pairs, axis=1)
    corr = float(np.corrcoef(a[0], a[1])[0, 1])
    want = 0.44 if direction == "forward" else -0.2
    assert abs(corr - want) < 0.05, corr


def test_local_search_normal_is_irwin_hall_12():
    # twelve 16-bit uniforms: mean 0, variance 1 (to 2^-32), excess kurtosis -6/60,
    # support [-6, 6); values are multiples of 2^-16
    z = np.array([o.ls_normal(5, 9, g, i, t, e) for g in range(2) for i in range(50)
                  for t in range(10) for e in range(20)])
    assert abs(z.mean()) < 5 / math.sqrt(len(z))
    assert abs(z.var() - 1.0) < 0.03
    kurt = np.mean((z - z.mean()) ** 4) / z.var() ** 2
    assert abs(kurt - 2.9) < 0.08
    assert np.all(np.abs(z) < 6) and np.all(np.round(z * 65536) == z * 65536)
    # distinct genes, iterations and individuals draw distinct values
    assert len(np.unique(z)) > 0.95 * len(z)
