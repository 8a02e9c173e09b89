"""The parity helpers' branch values: a pose within the margin of a score
discontinuity is compared against the score it would have on the other side.
These CPU tests check that the listed jumps are those changes, by moving the
pose across the grid face or the 8 A cutoff with the oracle alone."""
import numpy as np
import pytest

from helpers import MARGIN, OracleSide, branch_jumps, branch_ok, pairwise_jumps
from oracle import oracle as o
from paper_2509_12232_gb300 import synth


@pytest.fixture(scope="module")
def side():
    pk = synth.make_pocket(300, 6.0, seed=3)
    ligs = synth.LigandSet(
        atom_off=np.array([0, 1, 6], np.int32),
        x=np.array([0, 0.0, 1.5, 2.2, 3.7, 4.4], np.float32),
        y=np.array([0, 0.0, 0.0, 1.3, 1.3, 2.6], np.float32),
        z=np.zeros(6, np.float32),
        q=np.array([0.3, 0.3, 0, 0, 0, -0.2], np.float32),
        type=np.array([4, 0, 1, 2, 3, 6], np.uint8),
        parent=np.array([-1, -1, 0, 1, 2, 3], np.int16),
        tors_off=np.array([0, 0, 1], np.int32),
        tors_b=np.array([2], np.int16),
        ligand_id=np.array([1, 2], np.uint64))
    return OracleSide(pk, ligs)


def test_face_jump_is_the_change_across_the_face(side):
    g = side.grid
    hi = g.origin + (np.array(g.n) - 1) * g.h
    c = np.asarray(side.pk.center, np.float64)
    for d in (1e-5, -1e-5):   # just inside, just outside the far x face
        t = np.array([hi[0] - d, c[1] + 0.3, c[2] - 0.2]) - c
        geno = np.array([*t, 1, 0, 0, 0], np.float32)
        j = branch_jumps(side, 0, geno)
        assert len(j) == 1
        other = geno.copy()
        other[0] = np.float32(t[0] + 2 * d)          # the same atom on the other side
        s0 = side.score(0, geno[None])["score"][0]
        s1 = side.score(0, other[None])["score"][0]
        assert s0 + j[0] == pytest.approx(s1, abs=1e-3)
        assert branch_ok(s1, s0, j) and not branch_ok(s1, s0, [])
    far = np.array([0.5, 0.5, 0.5, 1, 0, 0, 0], np.float32)
    assert branch_jumps(side, 0, far) == []


def test_cutoff_jump_is_the_pair_term_at_8(side):
    lig = side.lig(1)
    P = side.P
    assert o.topology(lig)[1].tolist() == [[0, 4]]
    # atoms 0 and 4 (C, q 0.3 and ND, q -0.2) placed 8 A -+ 1e-5 apart
    for d in (1e-5, -1e-5):
        r = 8.0 - d
        xyz = np.zeros((5, 3))
        xyz[4, 0] = r
        j = pairwise_jumps(lig, P, o.PocketS([50.0], [50.0], [50.0], [0.0], [0], (0, 0, 0), 6.0),
                           xyz)
        assert len(j) == 1
        e_in = o.pair_terms(P, 0, 6, np.float32(0.3), np.float32(-0.2), 8.0 - 1e-9)[3]
        assert abs(j[0]) == pytest.approx(abs(e_in), rel=1e-4)  # the term at r, 1e-5 from 8
        assert np.sign(j[0]) == (-1 if r < 8 else 1) * np.sign(e_in)
    assert MARGIN > 1e-5
