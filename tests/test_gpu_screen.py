"""The chunked large screen (c5 settings: 10,000-atom pocket, 2,048 poses x
40 generations) on two chunks: the records of the chunked screen equal, bit
for bit, those of one dock_batch over both chunks; that search, traced, is
replayed against the oracle on sampled ligands of each chunk (GA bit-exact,
sampled FP32 scores within the bar, best records and FP64 rescores)."""
import math

import numpy as np
import pytest

from helpers import OracleSide, gpu_pocket, near_ok_grid, within
from oracle import oracle as o
from paper_2509_12232_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEARCH = dict(p_cross=0.8, p_mut=0.02)
CHUNK = 40


@pytest.fixture(scope="module")
def dock():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2509_12232_gb300 import build
    build.build()
    from paper_2509_12232_gb300 import dock as d
    return d


def _concat(a, b):
    n = lambda s: np.diff(s.atom_off)  # noqa: E731
    t = lambda s: np.diff(s.tors_off)  # noqa: E731
    return synth.LigandSet(
        atom_off=np.concatenate([[0], np.cumsum(np.r_[n(a), n(b)])]).astype(np.int32),
        x=np.r_[a.x, b.x], y=np.r_[a.y, b.y], z=np.r_[a.z, b.z], q=np.r_[a.q, b.q],
        type=np.r_[a.type, b.type], parent=np.r_[a.parent, b.parent],
        tors_off=np.concatenate([[0], np.cumsum(np.r_[t(a), t(b)])]).astype(np.int32),
        tors_b=np.r_[a.tors_b, b.tors_b], ligand_id=np.r_[a.ligand_id, b.ligand_id])


def test_two_chunk_screen_matches_one_batch_and_the_oracle(dock):
    from paper_2509_12232_gb300 import screen
    w = synth.WORKLOADS["c5"]
    pop, gens = w.pop, w.generations
    pk, _, _ = synth.make_workload("c5", n_ligands=0)
    chunks = [synth.screen_chunk("c5", c, size=CHUNK) for c in range(2)]
    assert int(chunks[1].ligand_id[0]) == CHUNK
    pocket = gpu_pocket(dock, pk)
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    recs, stats = screen.screen(pocket, chunks, pop, gens, seed=0, stream=stream, side_stream=side,
                                device=torch.cuda.current_device())
    assert [s[0] for s in stats] == [CHUNK, CHUNK]
    np.testing.assert_array_equal(recs["ligand_id"], np.arange(2 * CHUNK, dtype=np.uint64))
    assert np.all(recs["status"] == 0)
    # one batch over both chunks, traced
    ligs = _concat(*chunks)
    gl = screen._load(pocket, ligs, stream, None)
    goff = gl.geno_offsets(pop)
    tot = int(goff[-1])
    nl = ligs.n_ligands
    tg = torch.zeros(gens * tot, dtype=torch.float32, device="cuda")
    ts = torch.zeros(gens * nl * pop, dtype=torch.float32, device="cuda")
    job = dock.dock_batch(pocket, gl, pop, gens, seed=0, trace_genotypes=tg, trace_scores=ts,
                          stream=stream, **SEARCH)
    one = dock.dock_results(job)
    job.close()
    assert recs.tobytes() == one.tobytes()
    tg, ts = tg.cpu().numpy(), ts.cpu().numpy()
    side_o = OracleSide(pk, ligs)
    rng = np.random.default_rng(5)
    na = np.diff(ligs.atom_off)
    sample = [int(rng.integers(0, CHUNK)), int(np.argmax(na[:CHUNK])),
              CHUNK + int(rng.integers(0, CHUNK)), CHUNK + int(np.argmax(na[CHUNK:]))]
    for l in sample:
        k = ligs.n_tors(l)
        G = 7 + k
        lid = int(ligs.ligand_id[l])

        def geno(g):
            base = g * tot + int(goff[l])
            return tg[base: base + pop * G].reshape(pop, G)

        def scores(g):
            return ts[g * nl * pop + l * pop: g * nl * pop + (l + 1) * pop]

        for g in (0, 1, gens // 2, gens - 1):
            exp = o.ga_init(k, pop, pk.radius, 0, lid) if g == 0 else \
                o.ga_step(k, pop, SEARCH["p_cross"], SEARCH["p_mut"], 0, lid, g, geno(g - 1),
                          scores(g - 1))
            np.testing.assert_array_equal(geno(g).view(np.uint32), exp.view(np.uint32),
                                          err_msg="ligand %d generation %d" % (l, g))
            sel = rng.choice(pop, 24, replace=False)
            ref = side_o.score(l, geno(g)[sel])
            got = scores(g)[sel]
            ok = near_ok_grid(side_o, l, geno(g)[sel], got, ref["score"],
                              within(got, ref["score"]), ref["margin"] < 2e-4)
            assert ok.all(), (l, g, np.nonzero(~ok)[0][:5])
        fin = scores(gens - 1)
        key = [(np.inf if math.isnan(v) else v, i) for i, v in enumerate(fin.tolist())]
        order = [i for _, i in sorted(key)][:8]
        assert recs[l]["best_index"].tolist() == order
        ref = side_o.score(l, recs[l]["genotype"][:, :G])
        b64 = recs[l]["best_fp64"]
        assert np.all(near_ok_grid(side_o, l, recs[l]["genotype"][:, :G], b64, ref["score"],
                                   within(b64, ref["score"], rel=1e-5, abs_=1e-4),
                                   ref["margin"] < 2e-4, rel=1e-5, abs_=1e-4))
    gl.close()
