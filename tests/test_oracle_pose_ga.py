"""Pins of the oracle's pose application (Algorithm 1), ligand topology,
counter-based RNG and genetic algorithm.

Outside facts used: scipy's quaternion and rotation-vector routines, graph
distances and components from networkx, numpy's Philox4x64-10 bit generator,
rigid-body invariants (bond lengths, intra-fragment distances), the
equivalence of root-to-leaf and leaf-to-root torsion order and of rigid-first
and torsion-first order, Irwin-Hall moments, and GA invariants (elitism,
block crossover, unit quaternions, wrapped torsions, determinism).
"""
import math

import networkx as nx
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as o
from paper_2509_12232_gb300 import synth

P = o.Params(synth.TYPE_PARAMS)


def ligands(n=8, seed=21, sizes=(10, 40), tors=(1, 10)):
    rng = np.random.Generator(np.random.Philox(seed))
    na = rng.integers(sizes[0], sizes[1] + 1, size=n)
    nt = rng.integers(tors[0], tors[1] + 1, size=n)
    ls = synth.make_ligands(rng, na, nt)
    return [o.Ligand(**ls.ligand(i)) for i in range(n)]


def random_geno(rng, k):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    return np.concatenate([rng.uniform(-3, 3, 3), q, rng.uniform(-math.pi, math.pi, k)]).astype(np.float32)


# ---------------------------------------------------------------------------
def test_quaternion_matrix_matches_scipy():
    rng = np.random.default_rng(0)
    for _ in range(50):
        q = rng.normal(size=4)
        R = o.quat_matrix(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy: scalar last
        np.testing.assert_allclose(R, ref, atol=1e-14)


@pytest.mark.parametrize("lig", ligands())
def test_topology_matches_graph_library(lig):
    moves, pairs = o.topology(lig)
    par = lig.a["parent"]
    G = nx.Graph()
    G.add_nodes_from(range(lig.n))
    G.add_edges_from((int(par[i]), i) for i in range(1, lig.n))
    tb = [int(b) for b in lig.a["tors_b"]]
    for j, b in enumerate(tb):
        H = G.copy()
        H.remove_edge(int(par[b]), b)
        side = nx.node_connected_component(H, b) - {b}
        assert set(np.nonzero(moves[j])[0].tolist()) == side
    dist = dict(nx.all_pairs_shortest_path_length(G))
    F = G.copy()
    F.remove_edges_from((int(par[b]), b) for b in tb)
    frag = {}
    for fi, comp in enumerate(nx.connected_components(F)):
        for a in comp:
            frag[a] = fi
    expect = [[i, j] for i in range(lig.n) for j in range(i + 1, lig.n)
              if dist[i][j] > 3 and frag[i] != frag[j]]
    assert pairs.tolist() == expect


@pytest.mark.parametrize("lig", ligands())
def test_pose_preserves_bonds_and_fragments(lig):
    rng = np.random.default_rng(lig.n)
    x0 = np.stack([lig.a["x"], lig.a["y"], lig.a["z"]], 1).astype(np.float64)
    par = lig.a["parent"]
    tb = set(int(b) for b in lig.a["tors_b"])
    F = nx.Graph()
    F.add_nodes_from(range(lig.n))
    F.add_edges_from((int(par[i]), i) for i in range(1, lig.n) if i not in tb)
    d0 = np.linalg.norm(x0[:, None] - x0[None], axis=2)
    for _ in range(5):
        xyz = o.pose(lig, random_geno(rng, lig.k), [1.0, 2.0, 3.0])
        d = np.linalg.norm(xyz[:, None] - xyz[None], axis=2)
        for i in range(1, lig.n):
            assert d[i, par[i]] == pytest.approx(d0[i, par[i]], abs=1e-12)
        for comp in nx.connected_components(F):
            c = sorted(comp)
            np.testing.assert_allclose(d[np.ix_(c, c)], d0[np.ix_(c, c)], atol=1e-12)


@pytest.mark.parametrize("lig", ligands(seed=33))
def test_pose_invariant_pair_rule(lig):
    """The GPU path sums the included pairs whose distance no pose changes
    once per ligand: those where every torsion that moves one atom and not
    the other has the other on its axis. Checked here on the oracle's poses:
    such pairs keep their input distance, every other pair changes it."""
    moves, pairs = o.topology(lig)
    par = lig.a["parent"]
    axes = [(int(par[b]), int(b)) for b in lig.a["tors_b"]]

    def invariant(i, j):
        for t, (a, b) in enumerate(axes):
            if moves[t, i] != moves[t, j]:
                still = j if moves[t, i] else i
                if still not in (a, b):
                    return False
        return True

    x0 = np.stack([lig.a["x"], lig.a["y"], lig.a["z"]], 1).astype(np.float64)
    d0 = np.linalg.norm(x0[pairs[:, 0]] - x0[pairs[:, 1]], axis=1)
    rng = np.random.default_rng(lig.n + 3)
    dmax = np.zeros(len(pairs))
    for _ in range(8):
        xyz = o.pose(lig, random_geno(rng, lig.k), [0.0, 1.0, -2.0])
        d = np.linalg.norm(xyz[pairs[:, 0]] - xyz[pairs[:, 1]], axis=1)
        dmax = np.maximum(dmax, np.abs(d - d0))
    inv = np.array([invariant(int(i), int(j)) for i, j in pairs], bool)
    assert np.all(dmax[inv] < 1e-9)
    assert np.all(dmax[~inv] > 1e-4)


@pytest.mark.parametrize("lig", ligands())
def test_pose_orders_agree(lig):
    """Rigid-first (Algorithm 1's order), torsion-first, and leaf-to-root
    torsion order give the same geometry."""
    rng = np.random.default_rng(lig.n + 7)
    for _ in range(5):
        g = random_geno(rng, lig.k)
        a = o.pose(lig, g, [0.5, -1.0, 2.0], order=0)
        b = o.pose(lig, g, [0.5, -1.0, 2.0], order=1)
        c = o.pose(lig, g, [0.5, -1.0, 2.0], order=2)
        np.testing.assert_allclose(a, b, atol=1e-11)
        np.testing.assert_allclose(a, c, atol=1e-11)


@pytest.mark.parametrize("lig", ligands(4))
def test_identity_and_full_turn(lig):
    x0 = np.stack([lig.a["x"], lig.a["y"], lig.a["z"]], 1).astype(np.float64)
    c = np.array([3.0, -2.0, 0.5])
    ident = np.zeros(7 + lig.k, np.float32)
    ident[3] = 1.0
    np.testing.assert_allclose(o.pose(lig, ident, c), x0 - x0.mean(0) + c, atol=1e-12)
    turn = ident.copy()
    turn[7:] = np.float32(2 * math.pi)
    # float32(2 pi) differs from 2 pi by 1.7e-7 rad
    np.testing.assert_allclose(o.pose(lig, turn, c), x0 - x0.mean(0) + c, atol=1e-5)


def test_torsion_is_right_handed_rotation_about_bond():
    """With the identity rigid motion, torsion theta moves the fragment as the
    rotation vector theta * u (u along parent(b) -> b) about parent(b)."""
    lig = ligands(1, seed=5, sizes=(12, 12), tors=(1, 1))[0]
    moves, _ = o.topology(lig)
    b = int(lig.a["tors_b"][0])
    a = int(lig.a["parent"][b])
    x0 = np.stack([lig.a["x"], lig.a["y"], lig.a["z"]], 1).astype(np.float64)
    x0 = x0 - x0.mean(0)
    u = (x0[b] - x0[a]) / np.linalg.norm(x0[b] - x0[a])
    for theta in (0.3, -1.2, 2.9):
        g = np.array([0, 0, 0, 1, 0, 0, 0, theta], np.float32)
        xyz = o.pose(lig, g, [0, 0, 0])
        R = Rotation.from_rotvec(float(np.float32(theta)) * u).as_matrix()
        expect = x0.copy()
        expect[moves[0]] = (x0[moves[0]] - x0[a]) @ R.T + x0[a]
        np.testing.assert_allclose(xyz, expect, atol=1e-12)


def test_rigid_motion_matches_scipy():
    lig = ligands(1, seed=9)[0]
    x0 = np.stack([lig.a["x"], lig.a["y"], lig.a["z"]], 1).astype(np.float64)
    g = np.zeros(7 + lig.k, np.float32)
    g[:3] = [1.5, -2.25, 0.75]
    q = np.array([0.3, -0.5, 0.2, 0.7])
    q /= np.linalg.norm(q)
    g[3:7] = q
    xyz = o.pose(lig, g, [10, 20, 30])
    qq = g[3:7].astype(np.float64)
    R = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
    expect = (x0 - x0.mean(0)) @ R.T + np.array([10, 20, 30]) + g[:3].astype(np.float64)
    np.testing.assert_allclose(xyz, expect, atol=1e-12)


# ---------------------------------------------------------------------------
# RNG
# ---------------------------------------------------------------------------
def test_philox4x64_matches_numpy():
    """numpy's Philox is Philox4x64-10 and returns block (counter + 1)."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2 ** 63, size=4, dtype=np.int64)]
        key = [int(v) for v in rng.integers(0, 2 ** 63, size=2, dtype=np.int64)]
        bg = np.random.Philox(counter=ctr, key=key)
        ref = bg.random_raw(4)
        nxt = list(ctr)
        nxt[0] += 1
        np.testing.assert_array_equal(o.philox4x64(nxt, key), ref)


def test_rng_words_layout():
    w = o.rng_words(7, 11, 3, 5, 2)
    ref = o.philox4x64([2, 5, 3, 11], [7, 0])
    lo = (ref & 0xFFFFFFFF).astype(np.uint32)
    hi = (ref >> np.uint64(32)).astype(np.uint32)
    np.testing.assert_array_equal(w, np.stack([lo, hi], 1).ravel())


def test_irwin_hall_normal_moments():
    z = np.array([o.normal(1, 2, 3, i, 4) for i in range(40000)], np.float64)
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.03           # sum of 12 U(0,1) has variance exactly 1
    assert z.min() >= -6 and z.max() <= 6
    # kurtosis of Irwin-Hall(12) - 6 is 3 - 1.2/12 = 2.9
    k = ((z - z.mean()) ** 4).mean() / z.var() ** 2
    assert abs(k - 2.9) < 0.08


# ---------------------------------------------------------------------------
# GA
# ---------------------------------------------------------------------------
def test_ga_init_ranges_and_determinism():
    k, pop, R = 5, 512, 12.0
    g = o.ga_init(k, pop, R, 3, 77)
    assert np.all(g[:, :3] >= -R / 2) and np.all(g[:, :3] < R / 2)
    np.testing.assert_allclose(np.linalg.norm(g[:, 3:7].astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert np.all(g[:, 7:] >= -np.float32(math.pi)) and np.all(g[:, 7:] < np.float32(math.pi))
    np.testing.assert_array_equal(g, o.ga_init(k, pop, R, 3, 77))
    assert not np.array_equal(g, o.ga_init(k, pop, R, 4, 77))
    assert not np.array_equal(g, o.ga_init(k, pop, R, 3, 78))
    # translation is uniform: mean ~ 0, var ~ R^2 / 12
    assert abs(g[:, :3].mean()) < 0.3
    assert g[:, :3].var() == pytest.approx(R * R / 12, rel=0.1)


def test_ga_step_elitism_selection_and_invariants():
    k, pop = 6, 256
    rng = np.random.default_rng(4)
    prev = o.ga_init(k, pop, 12.0, 1, 5)
    sc = rng.normal(size=pop).astype(np.float32)
    nxt = o.ga_step(k, pop, 0.8, 0.02, 1, 5, 1, prev, sc)
    best = int(np.argmin(sc))
    np.testing.assert_array_equal(nxt[0], prev[best])
    np.testing.assert_allclose(np.linalg.norm(nxt[:, 3:7].astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert np.all(np.abs(nxt[:, 7:]) <= np.float32(math.pi))
    np.testing.assert_array_equal(nxt, o.ga_step(k, pop, 0.8, 0.02, 1, 5, 1, prev, sc))


def test_ga_no_crossover_no_mutation_copies_tournament_winners():
    k, pop = 3, 128
    prev = o.ga_init(k, pop, 12.0, 2, 9)
    sc = np.arange(pop, dtype=np.float32)[::-1].copy()   # lower index = worse
    nxt = o.ga_step(k, pop, 0.0, 0.0, 2, 9, 1, prev, sc)
    # every child is a copy of some parent, and selection favours good scores
    rows = {tuple(r) for r in prev.tolist()}
    assert all(tuple(r) in rows for r in nxt.tolist())
    idx = [next(i for i in range(pop) if np.array_equal(prev[i], r)) for r in nxt[1:]]
    # binary tournament: P(winner = i) grows with rank; mean score of winners
    # E[min of two uniforms] = 1/3 of the range
    assert np.mean(sc[idx]) == pytest.approx((pop - 1) / 3, rel=0.15)
    # check the tournament itself against the words
    for i in range(1, 20):
        w = o.rng_words(2, 9, 1, i, 0)
        a1, a2 = (int(w[0]) * pop) >> 32, (int(w[1]) * pop) >> 32
        win = a1 if (sc[a1] < sc[a2] or (sc[a1] == sc[a2] and a1 < a2)) else a2
        np.testing.assert_array_equal(nxt[i], prev[win])


def test_ga_crossover_moves_whole_blocks():
    k, pop = 4, 64
    prev = o.ga_init(k, pop, 12.0, 3, 1)
    sc = np.zeros(pop, np.float32)
    nxt = o.ga_step(k, pop, 1.0, 0.0, 3, 1, 2, prev, sc)
    for i in range(1, pop):
        w = o.rng_words(3, 1, 2, i, 0)
        a = min((int(w[0]) * pop) >> 32, (int(w[1]) * pop) >> 32)
        b = min((int(w[2]) * pop) >> 32, (int(w[3]) * pop) >> 32)
        B = 4 + k
        c1, c2 = (int(w[5]) * (B + 1)) >> 32, (int(w[6]) * (B + 1)) >> 32
        lo, hi = min(c1, c2), max(c1, c2)
        blocks = [0, 1, 2, 3, 3, 3, 3] + [4 + j for j in range(k)]
        exp = np.array([prev[b, g] if lo <= blocks[g] < hi else prev[a, g] for g in range(7 + k)],
                       np.float32)
        np.testing.assert_array_equal(nxt[i], exp)


def test_ga_mutation_rate_and_scale():
    k, pop = 10, 2048
    prev = o.ga_init(k, pop, 12.0, 4, 2)
    sc = np.zeros(pop, np.float32)
    nxt = o.ga_step(k, pop, 0.0, 0.02, 4, 2, 1, prev, sc)
    # with equal scores, tournament picks the lower index; compare to that parent
    diffs = 0
    total = 0
    for i in range(1, pop):
        w = o.rng_words(4, 2, 1, i, 0)
        a = min((int(w[0]) * pop) >> 32, (int(w[1]) * pop) >> 32)
        d = nxt[i, :3] - prev[a, :3]
        diffs += int(np.count_nonzero(d))
        total += 3
        assert np.all(np.abs(d) <= 6.0 + 1e-5)
    assert diffs / total == pytest.approx(0.02, abs=0.01)


def test_checkpoint_resume_is_bit_exact():
    """State = genotypes + scores per generation; a replayed step equals the
    uninterrupted one."""
    k, pop = 4, 128
    g0 = o.ga_init(k, pop, 12.0, 8, 3)
    s0 = np.random.default_rng(1).normal(size=pop).astype(np.float32)
    g1 = o.ga_step(k, pop, 0.8, 0.02, 8, 3, 1, g0, s0)
    saved = (g1.copy(), s0.copy())
    s1 = np.random.default_rng(2).normal(size=pop).astype(np.float32)
    g2 = o.ga_step(k, pop, 0.8, 0.02, 8, 3, 2, g1, s1)
    g2r = o.ga_step(k, pop, 0.8, 0.02, 8, 3, 2, saved[0], s1)
    np.testing.assert_array_equal(g2, g2r)


def test_free_run_best_never_worsens():
    pk, ligs, w = synth.make_workload("c1")
    pks = o.pocket_from(pk)
    grid = o.grid_build(pks, P)
    r1 = o.dock_batch(ligs, P, pks, grid, pop=64, generations=1, seed=0)
    r5 = o.dock_batch(ligs, P, pks, grid, pop=64, generations=6, seed=0)
    assert r5["best64"][0, 0] <= r1["best64"][0, 0] + 1e-9
    assert np.all(np.diff(r5["best64"][0]) >= -1e-6)    # best 8 sorted by FP32 score


def test_ga_mutation_scale_per_gene_class():
    """Every gene mutated (p_mut = 1), no crossover, all parents equal: each
    child's change is sigma z with z ~ N(0, 1) (Irwin-Hall), sigma = 1 A for the
    translation, 0.1 for each quaternion component and 0.5 rad for a torsion.
    The quaternion is renormalised after its step: from the identity parent
    (1, 0, 0, 0), component i of the child over component 0 is
    0.1 z_i / (1 + 0.1 z_0), whose standard deviation is 0.1 (1 + 0.03)^(1/2)
    to second order. Scales of 0.5, 2 or 0.05 times the right one fail."""
    k, pop = 6, 4096
    parent = np.zeros(7 + k, np.float32)
    parent[3] = 1.0
    parent[7:] = 0.25
    prev = np.tile(parent, (pop, 1))
    nxt = o.ga_step(k, pop, 0.0, 1.0, 21, 9, 3, prev, np.zeros(pop, np.float32))
    child = nxt[1:].astype(np.float64)
    dt = child[:, :3].ravel()
    assert np.std(dt) == pytest.approx(1.0, rel=0.03)
    assert abs(np.mean(dt)) < 0.05
    ratio = (child[:, 4:7] / child[:, 3:4]).ravel()
    assert np.std(ratio) == pytest.approx(0.1 * math.sqrt(1.03), rel=0.03)
    norms = np.linalg.norm(child[:, 3:7], axis=1)
    np.testing.assert_allclose(norms, 1.0, atol=1e-6)
    # parent torsions 0.25, steps at most 0.5 * 6 = 3 < pi: no wrap happens
    dth = (child[:, 7:] - 0.25).ravel()
    assert np.std(dth) == pytest.approx(0.5, rel=0.03)
    assert np.max(np.abs(dth)) <= 3.0 + 1e-6
    # elitism keeps individual 0 unchanged
    np.testing.assert_array_equal(nxt[0], parent)


def test_ga_torsion_wrap():
    """A torsion pushed past pi comes back by one turn of 2 pi_f."""
    k, pop = 2, 2048
    parent = np.zeros(9, np.float32)
    parent[3] = 1.0
    parent[7:] = np.float32(3.0)
    prev = np.tile(parent, (pop, 1))
    nxt = o.ga_step(k, pop, 0.0, 1.0, 5, 1, 1, prev, np.zeros(pop, np.float32))
    th = nxt[1:, 7:].astype(np.float64).ravel()
    assert np.all(th >= -np.pi - 1e-6) and np.all(th <= np.pi + 1e-6)
    wrapped = th < 0
    # P(3 + 0.5 z > pi) = P(z > 0.2832) = erfc(0.2832 / sqrt 2) / 2 = 0.3885
    assert wrapped.mean() == pytest.approx(0.5 * math.erfc((math.pi - 3.0) / (0.5 * math.sqrt(2))),
                                           abs=0.03)
    # a wrapped value is the unwrapped one minus 2 pi: it sits just above -pi
    assert np.all(th[wrapped] < -np.pi + 3.0)
