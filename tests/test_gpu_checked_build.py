"""The bounds-checked build (DOCK_CHECKED). Every index the search, local
search and pairwise kernels take from their inputs (pair records, slot rows,
torsion and moved-atom entries, grid records, cell-list ranges, work items,
selected individuals) is tested there; a failure writes the call's status
word and the host reports DOCK_EDEVICE, with no trap. This test builds
libdock_checked.so and runs parity tests against it in a child process (the
library is chosen when the binding first loads it): the c1 search replay
with graph and plain launches, forced lanes per pose, the Solis-Wets chain
replay and the pairwise scorer. They pass only if no check fails, since any
failure surfaces as a DockError."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_passes_the_replay_tests():
    from paper_2509_12232_gb300 import build
    lib = build.build(checked=True)
    assert lib.endswith("libdock_checked.so") and os.path.exists(lib)
    env = dict(os.environ, DOCK_CHECKED="1")
    sel = ("test_search_replay_c1 or test_search_forced_lanes or test_edge_ligands_ragged_population "
           "or test_standalone_chains_replay_bit_exact or test_pairwise_scores_match_oracle")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_gpu_parity.py", "tests/test_gpu_local_search.py",
                        "tests/test_gpu_pairwise.py", "-m", "gpu", "-k", sel],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout, tail


def test_checked_library_is_the_one_loaded_under_the_switch():
    env = dict(os.environ, DOCK_CHECKED="1")
    code = ("from paper_2509_12232_gb300 import dock; import os; "
            "print(os.path.basename(dock.LIB_PATH)); dock.lib()")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().splitlines()[0] == "libdock_checked.so"
