"""Pins of the oracle's pair terms, grid maps and scoring (Algorithm 2).

The paper prints no formulas; the oracle reads its terms as the AutoDock4
free-energy function (Section V: "functionally equivalent to the one in
AutoDock"). These tests tie that reading to facts outside the oracle's own
code: well positions and depths that the 12-6 and 12-10 forms fix, the
Gaussian's half-width, limits of the sigmoidal dielectric, bilinearity in the
charges, the exact split of the pair sum into per-type maps, exactness of
trilinear interpolation on linear fields and its textbook error bound, rigid
motion invariance of the pairwise form, and brute-force sums over pairs.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar
from scipy.spatial.transform import Rotation

from oracle import oracle as o
from paper_2509_12232_gb300 import synth

TP = synth.TYPE_PARAMS
P = o.Params(TP)
HB_PAIRS = [(6, 3), (6, 4), (6, 5), (3, 6), (4, 6), (5, 6)]
T = synth.N_TYPES


def non_hb_pairs():
    return [(i, j) for i in range(T) for j in range(T) if (i, j) not in HB_PAIRS]


@pytest.mark.parametrize("ti,tj", non_hb_pairs())
def test_lj_well_depth_and_position(ti, tj):
    R = 0.5 * (float(TP["Rii"][ti]) + float(TP["Rii"][tj]))
    eps = math.sqrt(float(TP["eps"][ti]) * float(TP["eps"][tj]))
    assert o.disp_raw(P, ti, tj, R) == pytest.approx(-eps, rel=1e-12)
    # zero crossing of a 12-6 well at R * 2^(-1/6)
    assert abs(o.disp_raw(P, ti, tj, R * 2 ** (-1 / 6))) < 1e-12
    res = minimize_scalar(lambda r: o.disp_raw(P, ti, tj, r), bounds=(0.8 * R, 1.5 * R),
                          method="bounded", options={"xatol": 1e-10})
    assert res.x == pytest.approx(R, rel=1e-5)
    # long-range tail of the 12-6 form is -2 eps (R/r)^6
    r = 40.0
    assert o.disp_raw(P, ti, tj, r) == pytest.approx(-2 * eps * (R / r) ** 6, rel=1e-6)


@pytest.mark.parametrize("ti,tj", HB_PAIRS)
def test_hbond_12_10_well(ti, tj):
    acc = ti if TP["hb_role"][ti] == synth.HB_ACCEPTOR else tj
    R, eps = float(TP["hb_R"][acc]), float(TP["hb_eps"][acc])
    assert o.disp_raw(P, ti, tj, R) == pytest.approx(-eps, rel=1e-12)
    # zero crossing of a 12-10 well: C/r^12 = D/r^10 at r^2 = 5 R^2 / 6
    assert abs(o.disp_raw(P, ti, tj, R * math.sqrt(5 / 6))) < 1e-12
    res = minimize_scalar(lambda r: o.disp_raw(P, ti, tj, r), bounds=(0.8 * R, 1.5 * R),
                          method="bounded", options={"xatol": 1e-10})
    assert res.x == pytest.approx(R, rel=1e-5)
    # the H-bond term replaces the 12-6 term and is weighted by the H-bond weight
    t = o.pair_terms(P, ti, tj, 0.0, 0.0, R)
    assert t[0] == pytest.approx(-0.1209 * eps, rel=1e-12)


def test_dielectric_limits_and_monotone():
    A, eps0, k = -8.5525, 78.4, 7.7839
    assert o.dielectric(0.0) == pytest.approx(A + (eps0 - A) / (1 + k), rel=1e-12)
    assert o.dielectric(1e6) == pytest.approx(eps0, rel=1e-12)
    r = np.linspace(0.01, 60, 500)
    e = np.array([o.dielectric(x) for x in r])
    assert np.all(np.diff(e) > 0)


def test_electrostatic_bilinear_and_sign():
    r = 4.2
    base = o.pair_terms(P, 0, 1, 0.3, 0.2, r)[1]
    assert base > 0                                   # like charges repel
    assert o.pair_terms(P, 0, 1, -0.3, 0.2, r)[1] == pytest.approx(-base, rel=1e-14)
    assert o.pair_terms(P, 0, 1, 0.6, 0.2, r)[1] == pytest.approx(2 * base, rel=1e-14)
    assert o.pair_terms(P, 0, 1, 0.0, 0.2, r)[1] == 0.0
    # electrostatic term times eps(r) r is constant in r
    for rr in (1.0, 2.5, 7.9):
        e = o.pair_terms(P, 0, 1, 0.3, 0.2, rr)[1]
        assert e * o.dielectric(rr) * rr == pytest.approx(base * o.dielectric(r) * r, rel=1e-12)


def test_desolvation_gaussian_half_width_and_symmetry():
    sigma = 3.6
    r_half = sigma * math.sqrt(2 * math.log(2))
    d0 = o.pair_terms(P, 2, 4, 0.1, -0.2, 1e-9 + 0.5)[2] / math.exp(-0.25 / (2 * sigma * sigma))
    dh = o.pair_terms(P, 2, 4, 0.1, -0.2, r_half)[2]
    assert dh == pytest.approx(0.5 * d0, rel=1e-9)
    # symmetric in the atoms: (S_i V_j + S_j V_i)
    a = o.pair_terms(P, 2, 4, 0.1, -0.2, 3.0)
    b = o.pair_terms(P, 4, 2, -0.2, 0.1, 3.0)
    np.testing.assert_allclose(a, b, rtol=1e-14)
    # charge dependence is through |q| only
    c = o.pair_terms(P, 2, 4, -0.1, 0.2, 3.0)
    assert c[2] == pytest.approx(a[2], rel=1e-14)


def test_cutoff_floor_and_cap():
    assert np.all(o.pair_terms(P, 0, 0, 0.4, 0.4, 8.0) == 0)
    assert np.all(o.pair_terms(P, 0, 0, 0.4, 0.4, 8.0 + 1e-9) == 0)
    assert o.pair_terms(P, 0, 0, 0.4, 0.4, 8.0 - 1e-9)[3] != 0
    np.testing.assert_array_equal(o.pair_terms(P, 1, 2, 0.4, -0.1, 0.1),
                                  o.pair_terms(P, 1, 2, 0.4, -0.1, 0.5))
    # raw 12-6 at r = 0.5 is far above the cap -> weighted cap
    assert o.disp_raw(P, 0, 0, 0.5) > 1e5
    assert o.pair_terms(P, 0, 0, 0.0, 0.0, 0.5)[0] == pytest.approx(0.1662 * 1e5, rel=1e-14)


def test_sum_of_terms():
    t = o.pair_terms(P, 3, 6, 0.25, -0.35, 3.1)
    assert t[3] == pytest.approx(t[0] + t[1] + t[2], rel=1e-15)


# ---------------------------------------------------------------------------
# Grid maps and trilinear lookup
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_pocket():
    pk = synth.make_pocket(300, 6.0, seed=3)
    return pk, o.pocket_from(pk)


@pytest.fixture(scope="module")
def small_grid(small_pocket):
    return o.grid_build(small_pocket[1], P)


def test_grid_geometry(small_grid, small_pocket):
    g = small_grid
    n = int(math.floor(2 * 6.0 / 0.375 + 1e-9)) + 1
    assert g.n == (n, n, n)
    np.testing.assert_allclose(g.origin + 0.5 * (n - 1) * 0.375, small_pocket[0].center, atol=1e-12)


def _one_atom_ligand(t, q, xyz):
    return o.Ligand(x=[xyz[0]], y=[xyz[1]], z=[xyz[2]], q=[q], type=[t], parent=[-1], tors_b=[])


def test_grid_equals_pairwise_at_nodes(small_grid, small_pocket):
    """At a node, M_t + q E + |q| D is the pair sum exactly (no cap active)."""
    g, (pk, pks) = small_grid, small_pocket
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(60):
        idx = rng.integers(0, g.n[0], size=3)
        xyz = g.origin + idx * g.h
        t = int(rng.integers(0, T))
        q = float(np.float32(rng.normal(0, 0.4)))
        if g.maps[t, idx[2], idx[1], idx[0]] >= 1e4:
            continue
        lig = _one_atom_ligand(t, q, xyz)
        eg, _ = o.inter_grid(lig, g, xyz[None, :])
        ep = o.inter_pairwise(lig, P, pks, xyz[None, :])
        assert eg == pytest.approx(ep, rel=1e-10, abs=1e-10)
        checked += 1
    assert checked > 30


def test_grid_node_matches_brute_force_sum(small_grid, small_pocket):
    g, (pk, pks) = small_grid, small_pocket
    idx = (5, 7, 3)
    p = g.origin + np.array(idx) * g.h
    for t in (0, 4, 6):
        tot = {"M": 0.0, "E": 0.0, "D": 0.0}
        for j in range(pk.n_atoms):
            r = float(np.linalg.norm(p - np.array([pk.x[j], pk.y[j], pk.z[j]], np.float64)))
            # one unit probe charge splits the terms: q=0 gives M_t, q=+1 minus q=0 gives E+D
            tq0 = o.pair_terms(P, t, pk.type[j], 0.0, pk.q[j], r)
            tot["M"] += tq0[3]
        assert g.maps[t, idx[2], idx[1], idx[0]] == pytest.approx(min(tot["M"], 1e5), rel=1e-10, abs=1e-12)
    E = sum(o.pair_terms(P, 0, pk.type[j], 1.0, pk.q[j], float(np.linalg.norm(
        p - np.array([pk.x[j], pk.y[j], pk.z[j]], np.float64))))[1] for j in range(pk.n_atoms))
    assert g.maps[T, idx[2], idx[1], idx[0]] == pytest.approx(E, rel=1e-10, abs=1e-12)


def test_trilinear_exact_on_linear_field(small_grid):
    g = small_grid
    nx, ny, nz = g.n
    X = g.origin[0] + np.arange(nx) * g.h
    Y = g.origin[1] + np.arange(ny) * g.h
    Z = g.origin[2] + np.arange(nz) * g.h
    f = (0.7 * X[None, None, :] - 1.3 * Y[None, :, None] + 0.25 * Z[:, None, None] + 2.0)
    grid = o.grid_with_maps(g.s, f[None])
    rng = np.random.default_rng(2)
    lo, hi = g.origin, g.origin + (np.array(g.n) - 1) * g.h
    for _ in range(200):
        p = rng.uniform(lo, hi)
        v = o.trilinear(grid, 0, *p)
        assert v == pytest.approx(0.7 * p[0] - 1.3 * p[1] + 0.25 * p[2] + 2.0, rel=1e-12, abs=1e-12)
    # faces: the far corner is inside, a hair beyond is outside
    assert o.trilinear(grid, 0, *hi) is not None
    assert o.trilinear(grid, 0, hi[0] + 1e-9, hi[1], hi[2]) is None
    assert o.trilinear(grid, 0, lo[0] - 1e-9, lo[1], lo[2]) is None


def test_trilinear_error_bound_smooth_field(small_grid):
    """|I f - f| <= h^2/8 (|f_xx| + |f_yy| + |f_zz|)max (tensor-product bound)."""
    g = small_grid
    nx, ny, nz = g.n
    X = g.origin[0] + np.arange(nx) * g.h
    Y = g.origin[1] + np.arange(ny) * g.h
    Z = g.origin[2] + np.arange(nz) * g.h
    a, b, c = 0.9, 0.6, 1.2
    f = np.sin(a * Z)[:, None, None] * np.cos(b * Y)[None, :, None] * np.sin(c * X)[None, None, :]
    grid = o.grid_with_maps(g.s, f[None])
    bound = g.h ** 2 / 8 * (a * a + b * b + c * c)
    rng = np.random.default_rng(3)
    lo, hi = g.origin, g.origin + (np.array(g.n) - 1) * g.h
    worst = 0.0
    for _ in range(400):
        p = rng.uniform(lo, hi)
        err = abs(o.trilinear(grid, 0, *p) - math.sin(a * p[2]) * math.cos(b * p[1]) * math.sin(c * p[0]))
        worst = max(worst, err)
    assert worst <= bound
    assert worst > bound / 50          # the bound is not vacuous here


def test_outside_atom_penalty(small_grid):
    g = small_grid
    hi = g.origin + (np.array(g.n) - 1) * g.h
    p = hi + np.array([0.5, 0.0, 0.0])
    lig = _one_atom_ligand(0, 0.1, p)
    e, m = o.inter_grid(lig, g, p[None, :])
    assert e == o.EOUT
    assert m == pytest.approx(0.0, abs=1e-12)   # on the y/z far faces


# ---------------------------------------------------------------------------
# Whole-ligand scoring
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1_small():
    rng = np.random.Generator(np.random.Philox(11))
    ligs = synth.make_ligands(rng, [14], [3])
    return o.Ligand(**ligs.ligand(0))


def test_joint_rigid_motion_invariance(c1_small, small_pocket):
    """A general joint rotation + translation of protein and ligand leaves the
    pairwise inter-energy unchanged up to the float32 rounding of the moved
    protein coordinates; intra is invariant under a ligand-only rigid motion."""
    lig = c1_small
    pk, pks = small_pocket
    xyz = o.pose(lig, [0.5, -0.3, 0.2, 0.8, 0.1, -0.3, 0.5, 0.4, -1.2, 2.0], pk.center)
    e_inter = o.inter_pairwise(lig, P, pks, xyz)
    e_intra, _ = o.intra(lig, P, xyz)
    R = Rotation.from_rotvec([0.3, -1.1, 0.7]).as_matrix()
    t = np.array([3.0, -7.5, 12.25])
    pxyz = np.stack([pk.x, pk.y, pk.z], 1).astype(np.float64) @ R.T + t
    moved = o.PocketS(pxyz[:, 0], pxyz[:, 1], pxyz[:, 2], pk.q, pk.type, pk.center, pk.radius)
    e_mov = o.inter_pairwise(lig, P, moved, xyz @ R.T + t)
    assert e_mov == pytest.approx(e_inter, rel=1e-5, abs=1e-4)
    e_intra2, _ = o.intra(lig, P, xyz @ R.T + t)
    assert e_intra2 == pytest.approx(e_intra, rel=1e-10, abs=1e-12)


def test_pairwise_inter_rigid_invariance_exact(c1_small):
    """Joint motion of ligand and protein with protein coords in float64 rounding-free form."""
    lig = c1_small
    rng = np.random.default_rng(5)
    prot = (np.round(rng.uniform(-10, 10, size=(80, 3)) * 64) / 64).astype(np.float32)
    types = rng.integers(0, T, 80).astype(np.uint8)
    qs = rng.normal(0, 0.4, 80).astype(np.float32)
    xyz = o.pose(lig, [0.1, 0.2, -0.3, 1, 0, 0, 0, 0.3, 0.9, -0.4], [0, 0, 0])
    pk = o.PocketS(prot[:, 0], prot[:, 1], prot[:, 2], qs, types, (0, 0, 0), 6.0)
    e0 = o.inter_pairwise(lig, P, pk, xyz)
    # a rotation by a multiple of 90 degrees plus an integer translation maps float32
    # coordinates to float32 coordinates exactly
    R = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], np.float64)
    t = np.array([4.0, -2.0, 1.0])
    p2 = (prot.astype(np.float64) @ R.T + t).astype(np.float32)
    pk2 = o.PocketS(p2[:, 0], p2[:, 1], p2[:, 2], qs, types, (0, 0, 0), 6.0)
    e1 = o.inter_pairwise(lig, P, pk2, xyz @ R.T + t)
    assert e1 == pytest.approx(e0, rel=1e-12, abs=1e-12)


def test_brute_force_pair_sums(c1_small, small_pocket):
    """inter_pairwise and intra equal explicit double loops over pair_terms."""
    import networkx as nx
    lig = c1_small
    pk, pks = small_pocket
    xyz = o.pose(lig, [1.0, 0.5, -0.5, 0.3, 0.4, 0.5, 0.6, 1.0, -2.0, 0.5], pk.center)
    e = 0.0
    for i in range(lig.n):
        for j in range(pk.n_atoms):
            r = np.linalg.norm(xyz[i] - np.array([pk.x[j], pk.y[j], pk.z[j]], np.float64))
            e += o.pair_terms(P, lig.a["type"][i], pk.type[j], lig.a["q"][i], pk.q[j], r)[3]
    assert o.inter_pairwise(lig, P, pks, xyz) == pytest.approx(e, rel=1e-12, abs=1e-12)
    G = nx.Graph()
    par = lig.a["parent"]
    G.add_edges_from((int(par[i]), i) for i in range(1, lig.n))
    rot = {(int(par[b]), int(b)) for b in lig.a["tors_b"]}
    e = 0.0
    for i in range(lig.n):
        for j in range(i + 1, lig.n):
            path = nx.shortest_path(G, i, j)
            edges = {(min(a, b), max(a, b)) for a, b in zip(path, path[1:])}
            if len(path) - 1 > 3 and edges & {(min(a, b), max(a, b)) for a, b in rot}:
                r = np.linalg.norm(xyz[i] - xyz[j])
                e += o.pair_terms(P, lig.a["type"][i], lig.a["type"][j], lig.a["q"][i],
                                  lig.a["q"][j], r)[3]
    assert o.intra(lig, P, xyz)[0] == pytest.approx(e, rel=1e-12, abs=1e-12)


def test_two_atom_and_three_atom_cases(small_grid):
    """A 2- or 3-atom chain has no pair beyond three bonds: intra is zero;
    its inter energy is the sum of one-atom lookups."""
    g = small_grid
    c = g.origin + 0.5 * (np.array(g.n) - 1) * g.h
    lig3 = o.Ligand(x=[c[0], c[0] + 1.5, c[0] + 2.2], y=[c[1], c[1], c[1] + 1.3], z=[c[2]] * 3,
                    q=[0.2, -0.1, -0.1], type=[0, 4, 6], parent=[-1, 0, 1], tors_b=[])
    xyz = np.stack([lig3.a["x"], lig3.a["y"], lig3.a["z"]], 1).astype(np.float64)
    assert o.intra(lig3, P, xyz)[0] == 0.0
    e3, _ = o.inter_grid(lig3, g, xyz)
    parts = sum(o.inter_grid(_one_atom_ligand(int(lig3.a["type"][i]), float(lig3.a["q"][i]),
                                              xyz[i]), g, xyz[i:i + 1])[0] for i in range(3))
    assert e3 == pytest.approx(parts, rel=1e-14)


def test_five_atom_chain_single_pair():
    """Chain 0-1-2-3-4 with a rotatable bond 1-2: the only included pair is
    (0, 4); its energy is the pair term at the posed distance."""
    x = [0.0, 1.5, 2.2, 3.7, 4.4]
    y = [0.0, 0.0, 1.3, 1.3, 2.6]
    lig = o.Ligand(x=x, y=y, z=[0.0] * 5, q=[0.3, 0, 0, 0, -0.2], type=[0, 1, 2, 3, 6],
                   parent=[-1, 0, 1, 2, 3], tors_b=[2])
    moves, pairs = o.topology(lig)
    assert pairs.tolist() == [[0, 4]]
    assert moves[0].tolist() == [False, False, False, True, True]
    for theta in (0.0, 1.0, 2.5):
        xyz = o.pose(lig, [0, 0, 0, 1, 0, 0, 0, theta], [0, 0, 0])
        r = np.linalg.norm(xyz[0] - xyz[4])
        e = o.pair_terms(P, 0, 6, np.float32(0.3), np.float32(-0.2), r)[3]
        assert o.intra(lig, P, xyz)[0] == pytest.approx(e, rel=1e-14)


# ---------------------------------------------------------------------------
# Energies worked by hand from the published constants
# ---------------------------------------------------------------------------
# Constants (AutoDock4 free-energy function): W_vdw 0.1662, W_hb 0.1209,
# W_elec 0.1406, Coulomb 332.06363, W_sol 0.1322, charge factor 0.01097,
# sigma 3.6 A; Mehler-Solmajer eps(r) = A + B / (1 + k exp(-lambda B r)) with
# A = -8.5525, B = 78.4 - A = 86.9525, k = 7.7839, lambda = 0.003627.
# Type parameters as the table stores them (float32): C  R 4.0, eps 0.15,
# V 33.51, solpar -0.00143; N  R 3.5, eps 0.16, V 22.45, solpar -0.00162;
# OA R 3.2, eps 0.2, V 17.16, solpar -0.00251, acceptor (R_hb 2.8,
# eps_hb 5.0); ND R 3.5, eps 0.16, V 22.45, solpar -0.00162, donor.
# The expected values below were worked out with a calculator from these
# numbers alone; a wrong weight, Coulomb constant, dielectric constant,
# Gaussian width or charge factor moves them far outside the tolerance.
HAND_REL = 1e-9

# C (q = +0.3) - OA (q = -0.2). At r = 3.0:
#   R = (4.0 + 3.2) / 2 = 3.6, eps = sqrt(0.15 * 0.2) = 0.173205085
#   (R/r)^6 = 1.2^6 = 2.985984, (R/r)^12 = 8.916101
#   vdW   = 0.1662 * 0.173205085 * (8.916101 - 2 * 2.985984)      =  0.0847518276
#   eps(3.0) = -8.5525 + 86.9525 / (1 + 7.7839 e^(-0.94611)) = 13.0665815
#   elec  = 0.1406 * 332.06363 * 0.3 * (-0.2) / (13.0665815 * 3.0)  = -0.0714619142
#   S_C = -0.00143 + 0.01097 * 0.3 = 0.001861, S_OA = -0.00251 + 0.01097 * 0.2 = -0.000316
#   desol = 0.1322 * (0.001861 * 17.16 - 0.000316 * 33.51) * e^(-9 / 25.92) = 0.00199408257
# r = 4.5 and 7.5 the same way (eps(4.5) = 21.6080016, eps(7.5) = 41.6784561).
HAND_C_OA = {
    3.0: (0.0847518275659137, -0.07146191420970993, 0.0019940825682854693),
    4.5: (-0.013114308112479827, -0.028809171270011997, 0.001291954646314351),
    7.5: (-0.0006998502190770031, -0.008961588449148133, 0.0003221517446985739),
}
# ND (donor, q = -0.1) - OA (acceptor, q = +0.25): the 12-10 form with the
# acceptor's R_hb = 2.8 and eps_hb = 5.0 in place of 12-6, weight W_hb:
#   r = 2.8 (the well): 0.1209 * (5 * 5 - 6 * 5) = -0.6045
#   r = 3.5: 0.1209 * (25 * 0.8^12 - 30 * 0.8^10) = -0.181741517
HAND_ND_OA = {
    2.8: (-0.6044999999999897, -0.034570216107120175, -0.00036684879328593946),
    3.5: (-0.18174151725421814, -0.021203327309545793, -0.0003094544371384055),
}


@pytest.mark.parametrize("r", sorted(HAND_C_OA))
def test_hand_worked_pair_energies_c_oa(r):
    t = o.pair_terms(P, 0, 4, 0.3, -0.2, r)
    vdw, el, ds = HAND_C_OA[r]
    assert t[0] == pytest.approx(vdw, rel=HAND_REL)
    assert t[1] == pytest.approx(el, rel=HAND_REL)
    assert t[2] == pytest.approx(ds, rel=HAND_REL)
    assert t[3] == pytest.approx(vdw + el + ds, rel=HAND_REL)


@pytest.mark.parametrize("r", sorted(HAND_ND_OA))
def test_hand_worked_pair_energies_hbond(r):
    vdw, el, ds = HAND_ND_OA[r]
    for ti, tj, qi, qj in ((6, 4, -0.1, 0.25), (4, 6, 0.25, -0.1)):  # either order
        t = o.pair_terms(P, ti, tj, np.float32(qi), np.float32(qj), r)
        assert t[0] == pytest.approx(vdw, rel=HAND_REL)
        assert t[1] == pytest.approx(el, rel=1e-7)   # charges rounded to float32
        assert t[2] == pytest.approx(ds, rel=1e-7)


def test_hand_worked_cap():
    """C-C at r = 1.0: the raw 12-6 value 0.15 (4^12 - 2 * 4^6) = 2,515,353.6
    is above the 1e5 cap, so the term is 0.1662 * 1e5 = 16,620."""
    t = o.pair_terms(P, 0, 0, np.float32(0.1), np.float32(0.1), 1.0)
    assert o.disp_raw(P, 0, 0, 1.0) == pytest.approx(2515353.6, rel=1e-7)
    assert t[0] == pytest.approx(16620.0, rel=1e-12)
    assert t[1] == pytest.approx(0.10451006276147873, rel=1e-7)
    assert t[2] == pytest.approx(-0.0028387348615425963, rel=1e-7)


def test_hand_worked_three_atom_ligand_with_one_torsion():
    """A 3-atom chain C-OA-ND with the bond 0-1 rotatable, posed by hand.

    Input atoms (0, 0, 0), (1.5, 0, 0), (3, 1.5, 0), centroid (1.5, 0.5, 0).
    Genotype: t = (1, 2, -0.5), q = (1, 0, 0, 1) (90 degrees about z after
    normalising: (x, y, z) -> (-y, x, z)), theta = pi/2, pocket centre 0.
    Rigid motion: R (x - c) + t gives (1.5, 0.5, -0.5), (1.5, 2, -0.5),
    (0, 3.5, -0.5). The torsion turns atom 2 by +90 degrees about the axis
    0 -> 1 (+y, right hand: (x, y, z) -> (z, y, -x) relative to atom 0):
    (-1.5, 3, 0) -> (0, 3, 1.5), so atom 2 ends at (1.5, 3.5, 1.0).
    Intra: no pair is more than three bonds apart, so 0.
    Inter against an OA (q -0.4) at (1.5, 3.5, 4) and an N (q 0.3) at
    (-3, 0.5, -0.5); distances and pair sums (vdW/H-bond + elec + desolv):
      C -OA 5.408327: -0.0266800741583   C -N 4.5:      0.0188785676229
      OA-OA 4.743416:  0.0476088909293   OA-N 4.743416: -0.0426424907423
      ND-OA 3.0 (12-10, H-bond): -0.54317659352   ND-N 5.612486: 0.00662980631573
    total -0.539381893553."""
    lig = o.Ligand(x=[0.0, 1.5, 3.0], y=[0.0, 0.0, 1.5], z=[0.0] * 3, q=[0.2, -0.3, 0.1],
                   type=[0, 4, 6], parent=[-1, 0, 1], tors_b=[1])
    theta = np.float32(np.pi / 2)   # float32: cos(theta) = -4.4e-8
    xyz = o.pose(lig, [1.0, 2.0, -0.5, 1.0, 0.0, 0.0, 1.0, theta], [0.0, 0.0, 0.0])
    np.testing.assert_allclose(xyz, [[1.5, 0.5, -0.5], [1.5, 2.0, -0.5], [1.5, 3.5, 1.0]],
                               atol=1e-6)
    assert o.intra(lig, P, xyz)[0] == 0.0
    pk = o.PocketS([1.5, -3.0], [3.5, 0.5], [4.0, -0.5], [-0.4, 0.3], [4, 2], (0, 0, 0), 10.0)
    exact = np.array([[1.5, 0.5, -0.5], [1.5, 2.0, -0.5], [1.5, 3.5, 1.0]])
    assert o.inter_pairwise(lig, P, pk, exact) == pytest.approx(-0.539381893552913, rel=1e-9)
    assert o.inter_pairwise(lig, P, pk, xyz) == pytest.approx(-0.539381893552913, rel=1e-6)
