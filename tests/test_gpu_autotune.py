"""The autotuner of the search kernel's launch shape: it measures a table of
shapes, picks the fastest, and the tuned search still replays bit-exactly
against the oracle (uneven ligand sizes, the c3 size mix)."""
import numpy as np
import pytest

from helpers import OracleSide, gpu_ligands, gpu_pocket
from paper_2509_12232_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotune_picks_fastest_and_tuned_search_is_exact():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2509_12232_gb300 import build
    build.build()
    from paper_2509_12232_gb300 import dock
    import test_gpu_parity as tp
    pk, ligs, w = synth.make_workload("c3", n_ligands=400)
    pocket = gpu_pocket(dock, pk)
    gl = gpu_ligands(dock, pocket, ligs)
    res = dock.dock_autotune(pocket, gl, pop=256, generations=4, stream=torch.cuda.current_stream())
    ms = [r["ms_per_generation"] for r in res["table"]]
    assert len(ms) >= 6 and all(m > 0 for m in ms)
    assert res["best"] == int(np.argmin(ms))
    assert max(r["atoms_per_lane"] for r in res["table"]) * 8 >= int(np.diff(ligs.atom_off).max())
    side = OracleSide(pk, ligs)
    na = np.diff(ligs.atom_off)
    check = [int(np.argmax(na)), int(np.argmin(na)), 17, 211]
    tp._replay(dock, side, gl, pocket, pop=256, gens=3, seed=4, ligs_check=check, poses_per_gen=32)
