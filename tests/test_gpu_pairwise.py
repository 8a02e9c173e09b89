"""The pairwise inter-energy scorer (dock_score_pairwise) against the oracle's
pairwise form, and the invariance that form has and the grid form lacks: a
rigid motion of protein and ligand together leaves the score unchanged.

Bars as for the grid scorer: 1e-4 relative or 1e-3 absolute per pose; poses
with a ligand-protein or intra pair within 2e-4 A of the 8 A cutoff are
counted apart (FP32 and FP64 geometry may fall on opposite sides)."""
import numpy as np
import pytest

from helpers import MARGIN, PARAMS, branch_ok, gpu_ligands, pairwise_jumps, within
from oracle import oracle as o
from paper_2509_12232_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import to_dev  # noqa: E402


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
    rng = np.random.Generator(np.random.Philox(2024))
    ligs = synth.make_ligands(rng, np.array([24, 10, 41, 60]), np.array([4, 2, 8, 12]), id_base=500)
    pocket = dock.dock_create_pocket(pk.x, pk.y, pk.z, pk.q, pk.type, pk.center, pk.radius,
                                     pk.spacing, PARAMS)
    gl = gpu_ligands(dock, pocket, ligs)
    return dict(pk=pk, ligs=ligs, pocket=pocket, gl=gl, P=o.Params(PARAMS), pks=o.pocket_from(pk))


def _genos(k, n, seed, radius):
    g = o.ga_init(k, n, radius, seed, 31)
    out = np.zeros((n, 23), np.float32)
    out[:, :7 + k] = g
    out[: n // 2, :3] *= 1.7  # half of the poses pushed into the protein shell
    return out


def _oracle(setup, l, genos, prot_xyz):
    lig = o.Ligand(**setup["ligs"].ligand(l))
    k = lig.k
    score, inter, margin = [], [], []
    for g in genos:
        xyz = o.pose(lig, g[:7 + k], setup["pk"].center)
        e_inter = o.inter_pairwise(lig, setup["P"], setup["pks"], xyz)
        e_intra, m_intra = o.intra(lig, setup["P"], xyz)
        d = np.linalg.norm(xyz[:, None, :] - prot_xyz[None], axis=2)
        score.append(e_inter + e_intra)
        inter.append(e_inter)
        margin.append(min(m_intra, float(np.abs(d - 8.0).min())))
    return np.array(score), np.array(inter), np.array(margin)


def _gpu(dock, setup, pocket, l, genos):
    n = genos.shape[0]
    pl = torch.full((n,), l, dtype=torch.int32, device="cuda")
    sc = torch.zeros(n, dtype=torch.float32, device="cuda")
    dock.dock_score_pairwise(pocket, setup["gl"], pl, to_dev(torch, genos), sc)
    torch.cuda.synchronize()
    return sc.cpu().numpy()


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_pairwise_scores_match_oracle(dock, setup, l):
    pk = setup["pk"]
    prot = np.stack([pk.x, pk.y, pk.z], 1).astype(np.float64)
    genos = _genos(setup["ligs"].n_tors(l), 160, 40 + l, pk.radius)
    ref, inter, margin = _oracle(setup, l, genos, prot)
    got = _gpu(dock, setup, setup["pocket"], l, genos)
    near = margin < MARGIN
    ok = within(got, ref)
    lig = o.Ligand(**setup["ligs"].ligand(l))
    for i in np.nonzero(~ok & near)[0]:
        xyz = o.pose(lig, genos[i, :lig.n_genes], pk.center)
        ok[i] = branch_ok(got[i], ref[i], pairwise_jumps(lig, setup["P"], setup["pks"], xyz))
    assert np.all(ok), (np.nonzero(~ok)[0][:5], got[~ok][:5], ref[~ok][:5])
    # about 430 of a pose's ligand-protein distances per A lie near 8 A, so a
    # pair within the margin is expected in ~10-16% of the poses; there the two
    # sides may differ by one pair's energy at the cutoff (a branch value)
    assert near.mean() <= 0.3
    # most poses have protein atoms within the cutoff (the test is not vacuous)
    assert np.mean(np.abs(inter) > 1e-2) > 0.5


def test_pairwise_invariant_under_joint_rigid_motion(dock, setup):
    from scipy.spatial.transform import Rotation
    pk = setup["pk"]
    Q = Rotation.from_rotvec([0.7, -1.1, 0.4])
    s = np.array([3.25, -7.5, 1.125])
    rot = lambda v: Q.apply(np.asarray(v, np.float64)) + s  # noqa: E731
    xyz = rot(np.stack([pk.x, pk.y, pk.z], 1))
    c2 = rot(np.asarray(pk.center, np.float64)[None])[0]
    pocket2 = dock.dock_create_pocket(xyz[:, 0].astype(np.float32), xyz[:, 1].astype(np.float32),
                                      xyz[:, 2].astype(np.float32), pk.q, pk.type,
                                      c2.astype(np.float32), pk.radius, pk.spacing, PARAMS)
    qQ = Q.as_quat()[[3, 0, 1, 2]]  # (w, x, y, z)

    def qmul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b.T
        return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)
    for l in range(4):
        g = _genos(setup["ligs"].n_tors(l), 128, 90 + l, pk.radius)
        g2 = g.copy()
        g2[:, :3] = Q.apply(g[:, :3].astype(np.float64))
        q = g[:, 3:7].astype(np.float64)
        g2[:, 3:7] = qmul(qQ, q / np.linalg.norm(q, axis=1, keepdims=True))
        a = _gpu(dock, setup, setup["pocket"], l, g)
        b = _gpu(dock, setup, pocket2, l, g2)
        ok = within(b, a)
        assert ok.mean() >= 0.99, (l, np.nonzero(~ok)[0][:5], a[~ok][:5], b[~ok][:5])


def test_pairwise_bad_ligand_index_scores_nan(dock, setup):
    pl = torch.tensor([0, 9, -1, 3], dtype=torch.int32, device="cuda")
    g = to_dev(torch, _genos(12, 4, 5, setup["pk"].radius))
    sc = torch.zeros(4, dtype=torch.float32, device="cuda")
    dock.dock_score_pairwise(setup["pocket"], setup["gl"], pl, g, sc)
    torch.cuda.synchronize()
    v = sc.cpu().numpy()
    assert np.isfinite(v[0]) and np.isfinite(v[3]) and np.isnan(v[1]) and np.isnan(v[2])
