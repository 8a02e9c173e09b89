"""Per-configuration precision of the FP32 search scores against the FP64
oracle (the compensated-sum FP32 scoring and the FP64 rescoring of the best
8 poses, checked and stated per configuration).

For each configuration a subset of its ligands runs the configuration's own
population and generation count through dock_batch (graph launch, default
lane shapes, as the benchmark runs it) with traced populations. Poses sampled
at the first, middle and last generation are rescored by the oracle: every
pose off a score discontinuity must meet the bar |E32 - E64| <= max(1e-3,
1e-4 |E64|), and the best-8 FP64 rescores must be within 1e-5 relative or
1e-4 absolute (the GPU interpolates FP32 maps, the oracle FP64 maps). Each test prints one
"precision" JSON line with the error distribution (run pytest with -s to see
it; DOCK_PRECISION_OUT, if set, names a file the lines are appended to).
"""
import json
import os

import numpy as np
import pytest

from helpers import MARGIN, OracleSide, branch_jumps, branch_ok, gpu_ligands, gpu_pocket, within
from paper_2509_12232_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEARCH = dict(p_cross=0.8, p_mut=0.02)
# configuration -> ligands of its own draw checked here
SUBSET = {"c1": 1, "c2": 24, "c3": 48, "c5": 16}


@pytest.fixture(scope="module")
def dock():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2509_12232_gb300 import build
    build.build()
    from paper_2509_12232_gb300 import dock as d
    d.lib()
    return d


def _report(line):
    s = json.dumps(line)
    print("\nprecision " + s)
    out = os.environ.get("DOCK_PRECISION_OUT")
    if out:
        with open(out, "a") as f:
            f.write(s + "\n")


@pytest.mark.parametrize("cfg", sorted(SUBSET))
def test_search_score_precision(dock, cfg):
    pk, ligs, w = synth.make_workload(cfg, n_ligands=SUBSET[cfg])
    side = OracleSide(pk, ligs)
    pocket = gpu_pocket(dock, pk)
    gl = gpu_ligands(dock, pocket, ligs)
    pop, gens, nl = w.pop, w.generations, ligs.n_ligands
    goff = gl.geno_offsets(pop)
    tot = int(goff[-1])
    tg = torch.zeros(gens * tot, dtype=torch.float32, device="cuda")
    ts = torch.zeros(gens * nl * pop, dtype=torch.float32, device="cuda")
    job = dock.dock_batch(pocket, gl, pop, gens, seed=0, use_graph=1, trace_genotypes=tg,
                          trace_scores=ts, stream=torch.cuda.current_stream(), **SEARCH)
    res = dock.dock_results(job)
    job.close()
    tg, ts = tg.cpu().numpy(), ts.cpu().numpy()
    rng = np.random.default_rng(17)
    e32, e64, near, near_ok = [], [], 0, 0
    r64_bar = 0.0
    for l in range(nl):
        G = 7 + ligs.n_tors(l)
        for g in sorted({0, gens // 2, gens - 1}):
            base = g * tot + int(goff[l])
            genos = tg[base: base + pop * G].reshape(pop, G)
            sc = ts[g * nl * pop + l * pop: g * nl * pop + (l + 1) * pop]
            sel = rng.choice(pop, min(pop, 64), replace=False)
            ref = side.score(l, genos[sel])
            far = ref["margin"] >= MARGIN
            for i in np.nonzero(~far)[0]:
                near += 1
                near_ok += int(branch_ok(float(sc[sel[i]]), ref["score"][i],
                                         branch_jumps(side, l, genos[sel[i]])))
            e32.append(sc[sel][far].astype(np.float64))
            e64.append(ref["score"][far])
        r = res[l]
        ref = side.score(l, r["genotype"][:, :G])
        far = ref["margin"] >= MARGIN
        over = np.abs(r["best_fp64"] - ref["score"]) / np.maximum(1e-4,
                                                                  1e-5 * np.abs(ref["score"]))
        r64_bar = max(r64_bar, float(over[far].max()) if far.any() else 0.0)
        ok64 = within(r["best_fp64"], ref["score"], rel=1e-5, abs_=1e-4)
        for i in np.nonzero(~ok64 & ~far)[0]:
            ok64[i] = branch_ok(r["best_fp64"][i], ref["score"][i],
                                branch_jumps(side, l, r["genotype"][i, :G]), rel=1e-5, abs_=1e-4)
        assert np.all(ok64), l
    e32, e64 = np.concatenate(e32), np.concatenate(e64)
    err = np.abs(e32 - e64)
    bar = np.maximum(1e-3, 1e-4 * np.abs(e64))
    ok = err <= bar
    n = int(err.size)
    line = {"config": cfg, "ligands": nl, "pop": pop, "generations": gens,
            "poses_checked": n, "poses_near_discontinuity": near,
            "near_poses_within_bar": near_ok,
            "abs_err_median": float(np.median(err)), "abs_err_p99": float(np.quantile(err, 0.99)),
            "abs_err_max": float(err.max()),
            "rel_err_max": float((err / np.maximum(1.0, np.abs(e64))).max()),
            "err_over_bar_max": float((err / bar).max()),
            "score_median": float(np.median(e64)),
            "score_range": [float(e64.min()), float(e64.max())],
            "fp64_rescore_err_over_bar_max": r64_bar, "within_bar": int(ok.sum())}
    _report(line)
    assert np.all(ok), (cfg, np.nonzero(~ok)[0][:5], e32[~ok][:5], e64[~ok][:5])
    # a pose within 2e-4 A of a grid face or of the 8 A cutoff may take the
    # other branch in FP32; such poses must stay rare (about 1% of them here),
    # and each must meet the bar against one of its branch values
    assert near <= max(2, (n + near) // 50)
    assert near_ok == near, (cfg, near, near_ok)
