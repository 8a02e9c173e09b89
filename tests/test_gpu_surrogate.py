"""GPU parity of the learned pre-screen: features, the BF16 MLP's forward and
backward against the FP64 oracle, training, and the pre-screened search.

Bars: features within one BF16 step of the oracle's FP64 values rounded to
BF16 (poses with an atom within 1e-4 A of a shell boundary excluded); MLP
gradients within 2e-2 relative (norm per tensor) of the FP64 oracle run on
the same BF16-rounded weights and inputs; predictions within 2e-2 of the
output scale; pre-screened generations bit-exact against the oracle's GA,
top-k and merge fed the GPU's predictions and scores.
"""
import math

import numpy as np
import pytest

from helpers import OracleSide, branch_jumps, compare_scores, gpu_ligands, gpu_pocket, within
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
def env(dock):
    pk, _, _ = synth.make_workload("c1")
    rng = np.random.Generator(np.random.Philox(77))
    ligs = synth.make_ligands(rng, [24, 12, 41, 30, 9], [4, 3, 9, 6, 1], id_base=300)
    side = OracleSide(pk, ligs)
    pocket = gpu_pocket(dock, pk)
    gl = gpu_ligands(dock, pocket, ligs)
    return dict(pk=pk, ligs=ligs, side=side, pocket=pocket, gl=gl)


def bf16_to_f64(u16):
    return (np.asarray(u16, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def shell_margin(xyz, center, R):
    d = np.linalg.norm(xyz - center, axis=-1)
    w = R / 8
    b = np.arange(1, 8) * w
    return np.abs(d[..., None] - b).min(axis=(-1, -2))


def test_features_and_scores_match_oracle(dock, env):
    side, ligs = env["side"], env["ligs"]
    rows, lig_of, refs, margins, scores_ref, smargin = [], [], [], [], [], []
    for l in range(ligs.n_ligands):
        lig = side.lig(l)
        g = o.ga_init(lig.k, 96, env["pk"].radius, 5 + l, 123)
        r = side.score(l, g, want_xyz=True)
        for i in range(g.shape[0]):
            row = np.zeros(23, np.float32)
            row[:lig.n_genes] = g[i]
            rows.append(row)
            lig_of.append(l)
            refs.append(o.to_bf16(o.features(lig, r["xyz"][i], env["pk"].center, g[i], env["pk"].radius)))
        margins.append(shell_margin(r["xyz"], np.asarray(env["pk"].center), env["pk"].radius))
        scores_ref.append(r["score"])
        smargin.append(r["margin"])
    genos = np.array(rows)
    n = genos.shape[0]
    dg = to_dev(torch, genos)
    pl = to_dev(torch, np.array(lig_of, np.int32))
    feats = torch.zeros(n, 128, dtype=torch.int16, device="cuda")
    sc = torch.zeros(n, dtype=torch.float32, device="cuda")
    dock.dock_features(env["pocket"], env["gl"], pl, dg, feats, scores=sc)
    torch.cuda.synchronize()
    got = bf16_to_f64(feats.cpu().numpy().view(np.uint16))
    ref = np.array(refs)
    margin = np.concatenate(margins)
    ok_rows = margin >= 1e-4
    assert ok_rows.mean() > 0.97
    tol = 2.0 ** -7 * np.abs(ref) + 1e-4
    bad = (np.abs(got - ref) > tol) & ok_rows[:, None]
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], ref[bad][:5])
    c, near, worst, fails = compare_scores(
        sc.cpu().numpy(), np.concatenate(scores_ref), np.concatenate(smargin),
        lambda i: branch_jumps(side, lig_of[i], genos[i, :side.lig(lig_of[i]).n_genes]))
    assert len(fails) == 0


def oracle_params(p32):
    """The oracle's view of the GPU network: W1..W3 as their BF16 copies, the
    rest as the FP32 masters."""
    p = p32.astype(np.float64)
    W1, b1, W2, b2, W3, b3, W4, b4 = o.mlp_unpack(p)
    for W in (W1, W2, W3):
        W[...] = o.to_bf16(W)
    return p


@pytest.fixture(scope="module")
def feature_rows(dock, env):
    """Realistic BF16 feature rows: features of random poses of the test ligands."""
    ligs = env["ligs"]
    rows, lig_of = [], []
    for l in range(ligs.n_ligands):
        k = ligs.n_tors(l)
        g = o.ga_init(k, 80, env["pk"].radius, 50 + l, 9)
        for i in range(g.shape[0]):
            row = np.zeros(23, np.float32)
            row[:7 + k] = g[i]
            rows.append(row)
            lig_of.append(l)
    n = len(rows)
    feats = torch.zeros(n, 128, dtype=torch.int16, device="cuda")
    dock.dock_features(env["pocket"], env["gl"], to_dev(torch, np.array(lig_of, np.int32)),
                       to_dev(torch, np.array(rows)), feats)
    torch.cuda.synchronize()
    return feats


@pytest.mark.parametrize("rows", [256, 4096])
def test_mlp_gradients_match_oracle(dock, feature_rows, rows):
    """Gradients of one batch against the oracle's FP64 backward: 256 rows of
    realistic features, and a full training batch (4,096 rows: 32 row tiles
    per product, the split-K weight gradients at their training split)."""
    S = dock.dock_surrogate_create(seed=3)
    if rows <= feature_rows.shape[0]:
        X = feature_rows[:rows]
    else:
        g = torch.Generator(device="cuda").manual_seed(rows)
        X = (torch.randn(rows, 128, device="cuda", generator=g) * 0.5).to(torch.bfloat16)
        X = X.view(torch.int16)
    t = np.random.default_rng(4).normal(size=X.shape[0]).astype(np.float32)
    grad = torch.zeros(dock.DOCK_MLP_N_PARAMS, dtype=torch.float32, device="cuda")
    loss = dock.dock_surrogate_gradients(S, X, to_dev(torch, t), grad)
    p32, _, _, _ = dock.dock_surrogate_get_params(S)
    P = oracle_params(p32)
    Xf = bf16_to_f64(X.cpu().numpy().view(np.uint16))
    loss_ref, g_ref = o.mlp_backward(P, Xf, t.astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    g = grad.cpu().numpy().astype(np.float64)
    for name, a, b in zip(["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"], o.mlp_unpack(g),
                          o.mlp_unpack(g_ref)):
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        assert rel <= 2e-2, (name, rel)


def test_mlp_predict_matches_oracle(dock, feature_rows):
    S = dock.dock_surrogate_create(seed=5)
    p32, _, _, _ = dock.dock_surrogate_get_params(S)
    dock.dock_surrogate_set_params(S, p32, t_mean=0.0, t_std=1.0)
    X = feature_rows
    out = torch.zeros(X.shape[0], dtype=torch.float32, device="cuda")
    dock.dock_surrogate_predict(S, X, out)
    torch.cuda.synchronize()
    ref = o.mlp_forward(oracle_params(p32), bf16_to_f64(X.cpu().numpy().view(np.uint16)))
    got = out.cpu().numpy()
    scale = np.sqrt(np.mean(ref ** 2)) + 1e-6
    assert np.max(np.abs(got - ref)) <= 2e-2 * (np.abs(ref) + scale).max()
    assert np.corrcoef(got, ref)[0, 1] > 0.999


@pytest.mark.parametrize("n", [1, 127, 129, 50_001, 400_001, 4_194_304])
def test_mlp_predict_tiles_and_ragged_tail(dock, n):
    """The fused tensor-core forward pass over many 128-row tiles per CTA
    (400,001 rows give every CTA about ten rounds of its two tile slots;
    4,194,304 is the benchmark's pre-screened generation, sampled) and
    a ragged last tile: every sampled row equals the oracle's network within
    the BF16 budget, no row is left unwritten, a second call gives the same
    bits, and the result does not depend on how the rows are batched."""
    S = dock.dock_surrogate_create(seed=11)
    p32, _, _, _ = dock.dock_surrogate_get_params(S)
    dock.dock_surrogate_set_params(S, p32, t_mean=1.5, t_std=2.0)
    g = torch.Generator(device="cuda").manual_seed(n)
    X = (torch.randn(n, 128, device="cuda", generator=g) * 0.7).to(torch.bfloat16).view(torch.int16)
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    dock.dock_surrogate_predict(S, X, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    again = torch.zeros(n, dtype=torch.float32, device="cuda")
    dock.dock_surrogate_predict(S, X, again)
    torch.cuda.synchronize()
    assert np.array_equal(again.cpu().numpy(), got)
    rows = np.unique(np.concatenate([np.arange(min(n, 64)), np.arange(max(0, n - 64), n),
                                     np.random.default_rng(n).integers(0, n, 256)]))
    ref = o.mlp_forward(oracle_params(p32), bf16_to_f64(X[rows].cpu().numpy().view(np.uint16)))
    ref = ref * 2.0 + 1.5
    scale = np.sqrt(np.mean(ref ** 2)) + 1e-6
    assert np.max(np.abs(got[rows] - ref)) <= 2e-2 * (np.abs(ref) + scale).max()
    if n > 200:
        part = torch.zeros(200, dtype=torch.float32, device="cuda")
        dock.dock_surrogate_predict(S, X[n - 200:], part)
        torch.cuda.synchronize()
        assert np.array_equal(part.cpu().numpy(), got[n - 200:])


def test_surrogate_search_replay(dock, env):
    """Pre-screened generations equal the oracle's GA children -> top-k of the
    GPU predictions -> merge with the GPU's exact scores, bit for bit."""
    side, ligs = env["side"], env["ligs"]
    pop, C, K, gens, seed = 48, 96, 20, 4, 7
    S = dock.dock_surrogate_create(seed=11)
    nl = ligs.n_ligands
    goff = env["gl"].geno_offsets(pop)
    tot = int(goff[-1])
    tg = torch.zeros(gens * tot, dtype=torch.float32, device="cuda")
    ts = torch.zeros(gens * nl * pop, dtype=torch.float32, device="cuda")
    job = dock.dock_batch(env["pocket"], env["gl"], pop, gens, seed=seed, trace_genotypes=tg,
                          trace_scores=ts, surrogate=S, candidates=C, keep=K,
                          stream=torch.cuda.current_stream(), **SEARCH)
    res = dock.dock_results(job)
    R = env["pk"].radius
    for l in range(nl):
        k = ligs.n_tors(l)
        G = 7 + k
        lid = int(ligs.ligand_id[l])

        def geno(g):
            return tg[g * tot + int(goff[l]): g * tot + int(goff[l]) + pop * G].cpu().numpy().reshape(pop, G)

        def scores(g):
            return ts[g * nl * pop + l * pop: g * nl * pop + (l + 1) * pop].cpu().numpy()

        np.testing.assert_array_equal(geno(0), o.ga_init(k, pop, R, seed, lid))
        for g in range(1, gens):
            kids = o.ga_children(k, pop, C, SEARCH["p_cross"], SEARCH["p_mut"], seed, lid, g,
                                 geno(g - 1), scores(g - 1))
            rows = np.zeros((C, 23), np.float32)
            rows[:, :G] = kids
            drows = to_dev(torch, rows)
            pl = torch.full((C,), l, dtype=torch.int32, device="cuda")
            feats = torch.zeros(C, 128, dtype=torch.int16, device="cuda")
            dock.dock_features(env["pocket"], env["gl"], pl, drows, feats)
            pred = torch.zeros(C, dtype=torch.float32, device="cuda")
            dock.dock_surrogate_predict(S, feats, pred)
            torch.cuda.synchronize()
            kept = o.topk(pred.cpu().numpy(), K)
            kept_rows = to_dev(torch, rows[kept])
            ksc = torch.zeros(K, dtype=torch.float32, device="cuda")
            dock.dock_score(env["pocket"], env["gl"], pl[:K], kept_rows, scores=ksc)
            torch.cuda.synchronize()
            ks = ksc.cpu().numpy()
            ref = side.score(l, kids[kept])
            c, near, worst, fails = compare_scores(ks, ref["score"], ref["margin"],
                                                   lambda i: branch_jumps(side, l, kids[kept][i]))
            assert len(fails) == 0
            origin, index = o.merge(scores(g - 1), ks, pop)
            kk, prev_g, prev_s = kids[kept], geno(g - 1), scores(g - 1)
            exp_g = np.array([kk[i] if og else prev_g[i] for og, i in zip(origin, index)])
            exp_s = np.array([ks[i] if og else prev_s[i] for og, i in zip(origin, index)], np.float32)
            np.testing.assert_array_equal(geno(g).view(np.uint32), exp_g.view(np.uint32),
                                          err_msg="ligand %d generation %d" % (l, g))
            np.testing.assert_array_equal(scores(g).view(np.uint32), exp_s.view(np.uint32))
        r = res[l]
        assert int(r["exact_evals"]) == pop + (gens - 1) * K
        assert int(r["surrogate_evals"]) == (gens - 1) * C
        ref = side.score(l, r["genotype"][:, :G])
        assert np.all(within(r["best_fp64"], ref["score"], rel=1e-5, abs_=1e-4) | (ref["margin"] < 2e-4))


def training_set(dock, pocket, pk, n_ligands, pop, gens, seed):
    """(features, exact scores) of every pose of plain GA trajectories."""
    rng = np.random.Generator(np.random.Philox(seed))
    na, nt = synth.ligand_sizes(rng, "uniform", n_ligands)
    ligs = synth.make_ligands(rng, na, nt, id_base=10_000 * seed)
    gl = gpu_ligands(dock, pocket, ligs)
    goff = gl.geno_offsets(pop)
    tot = int(goff[-1])
    tg = torch.zeros(gens * tot, dtype=torch.float32, device="cuda")
    job = dock.dock_batch(pocket, gl, pop, gens, seed=seed, trace_genotypes=tg,
                          stream=torch.cuda.current_stream(), **SEARCH)
    dock.dock_results(job)
    F = torch.zeros(gens * n_ligands * pop, 128, dtype=torch.int16, device="cuda")
    Y = torch.zeros(gens * n_ligands * pop, dtype=torch.float32, device="cuda")
    rows = n_ligands * pop
    for g in range(gens):
        dock.dock_features_population(pocket, gl, pop, tg[g * tot:(g + 1) * tot],
                                      F[g * rows:(g + 1) * rows], Y[g * rows:(g + 1) * rows])
    return F, Y, ligs, gl


def spearman(a, b):
    ra = np.argsort(np.argsort(a))
    rb = np.argsort(np.argsort(b))
    return np.corrcoef(ra, rb)[0, 1]


def test_training_learns_and_gains_over_random(dock, env):
    """Trained on exact scores of GA trajectories (per-pocket; held-out
    ligands drawn with another seed), the network (a) reduces its loss, (b)
    ranks held-out poses across ligands and generations (Spearman > 0.35),
    and (c) keeps the exact best of a population in its predicted best 10%
    more than twice as often as a random 10% does, averaged over the first
    three generations. Within a converged population the radial-shell
    features carry little signal (measured and reported, not asserted)."""
    pocket, pk = env["pocket"], env["pk"]
    F, Y, _, _ = training_set(dock, pocket, pk, n_ligands=256, pop=512, gens=16, seed=1)
    S = dock.dock_surrogate_create(seed=2)
    losses = dock.dock_surrogate_train(S, F, Y, epochs=3, batch=4096, lr=1e-3, score_clip=100.0)
    assert losses[-1] < 0.85 * losses[0], losses
    Fh, Yh, _, _ = training_set(dock, pocket, pk, n_ligands=32, pop=512, gens=6, seed=3)
    pred = torch.zeros(Fh.shape[0], dtype=torch.float32, device="cuda")
    dock.dock_surrogate_predict(S, Fh, pred)
    torch.cuda.synchronize()
    p, y = pred.cpu().numpy(), Yh.cpu().numpy()
    rows = 32 * 512
    report = {}
    for g in range(6):
        hits, rhos = 0, []
        for l in range(32):
            sl = slice(g * rows + l * 512, g * rows + (l + 1) * 512)
            yy, pp = y[sl], p[sl]
            keep = np.argsort(pp, kind="stable")[:52]
            hits += int(np.argmin(yy) in keep)
            rhos.append(spearman(pp, np.minimum(yy, 100.0)))
        report[g] = (round(float(np.median(rhos)), 3), hits / 32)
    glob = spearman(p, np.minimum(y, 100.0))
    print("held-out: global spearman %.3f; per generation (median within-ligand spearman, "
          "top-1 kept in the predicted best 10%%): %s" % (glob, report))
    assert glob > 0.35, glob
    assert np.mean([report[g][1] for g in range(3)]) > 0.2, report
