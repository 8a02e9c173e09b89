"""dock_batch_noalloc, the search entry point that allocates nothing.

Some callers cannot allocate GPU memory while they run: their device memory
belongs to another framework's pool, or a rule forbids cudaMalloc/cudaFree
after start-up. For them dock_batch_noalloc keeps every working buffer of the
search in one fixed device array inside the library. These tests call it
through the C ABI twice in a row (the array keeps the previous call's
contents) and check its results against dock_batch's, and that a search too
large for the array is refused with an error instead of running.
"""
import numpy as np
import pytest

from helpers import gpu_ligands, gpu_pocket, within
from paper_2509_12232_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2509_12232_gb300 import build
    build.build()
    from paper_2509_12232_gb300 import dock
    pk, _, _ = synth.make_workload("c1")
    rng = np.random.Generator(np.random.Philox(42))
    ligs = synth.make_ligands(rng, [24, 9, 40, 3], [4, 2, 7, 0], id_base=900)
    pocket = gpu_pocket(dock, pk)
    gl = gpu_ligands(dock, pocket, ligs)
    return dock, pocket, gl, ligs


def test_noalloc_matches_dock_batch_on_two_calls(setup):
    dock, pocket, gl, ligs = setup
    stream = torch.cuda.current_stream()
    pop, gens, seed = 160, 6, 5
    ref = dock.dock_results(dock.dock_batch(pocket, gl, pop, gens, seed=seed, use_graph=0,
                                            stream=stream))
    n = ligs.n_ligands
    out = torch.empty(n * dock.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for call in range(2):
        out.fill_(0xAB)            # stale bytes must all be overwritten
        dock.dock_batch_noalloc(pocket, gl, out, pop, gens, seed=seed, stream=stream)
        torch.cuda.synchronize()
        res = out.cpu().numpy().view(dock.RESULT_DTYPE)
        np.testing.assert_array_equal(res["ligand_id"], ref["ligand_id"])
        np.testing.assert_array_equal(res["n_genes"], ref["n_genes"])
        np.testing.assert_array_equal(res["status"], 0)
        np.testing.assert_array_equal(res["best_index"], ref["best_index"])
        np.testing.assert_array_equal(res["exact_evals"], ref["exact_evals"])
        assert np.all(within(res["best_fp32"], ref["best_fp32"]))
        assert np.all(within(res["best_fp64"], ref["best_fp64"], rel=1e-5, abs_=1e-4))
        np.testing.assert_allclose(res["genotype"], ref["genotype"], rtol=0, atol=1e-6)


def test_noalloc_refuses_searches_larger_than_its_array(setup):
    dock, pocket, gl, _ = setup
    stream = torch.cuda.current_stream()
    rng = np.random.Generator(np.random.Philox(43))
    big = gpu_ligands(dock, pocket, synth.make_ligands(rng, [12] * 60, [2] * 60))
    out = torch.empty(65 * dock.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    # 60 ligands x 4,096 poses x 9 genes x 2 buffers is about 17 MB of scratch
    with pytest.raises(dock.DockError) as e:
        dock.dock_batch_noalloc(pocket, big, out, 4096, 3, stream=stream)
    assert e.value.status == dock.DOCK_EINVAL
    assert "bytes of scratch" in str(e.value)
    too_many = gpu_ligands(dock, pocket, synth.make_ligands(rng, [8] * 65, [1] * 65))
    with pytest.raises(dock.DockError) as e:
        dock.dock_batch_noalloc(pocket, too_many, out, 16, 2, stream=stream)
    assert e.value.status == dock.DOCK_EINVAL
    # the library stays usable
    dock.dock_batch_noalloc(pocket, gl, out, 64, 2, stream=stream)
    torch.cuda.synchronize()


def test_noalloc_refuses_a_results_buffer_too_small(setup):
    """The kernels write one record per ligand into the caller's buffer; the
    wrapper refuses a buffer that cannot hold them, or one on the host."""
    dock, pocket, gl, ligs = setup
    stream = torch.cuda.current_stream()
    one = torch.empty(dock.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    with pytest.raises(dock.DockError) as e:
        dock.dock_batch_noalloc(pocket, gl, one, 64, 2, stream=stream)
    assert e.value.status == dock.DOCK_EINVAL
    host = torch.empty(ligs.n_ligands * dock.RESULT_DTYPE.itemsize, dtype=torch.uint8)
    with pytest.raises(dock.DockError) as e:
        dock.dock_batch_noalloc(pocket, gl, host, 64, 2, stream=stream)
    assert e.value.status == dock.DOCK_EINVAL


def test_noalloc_deadline_reaches_every_record_and_does_not_carry_over(setup):
    """A deadline that has passed before the first work item stops the search;
    every record reports DOCK_ETIMEOUT. The status words live in the shared
    array and are cleared per call, so the next call reports 0."""
    dock, pocket, gl, ligs = setup
    stream = torch.cuda.current_stream()
    n = ligs.n_ligands
    out = torch.empty(n * dock.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    dock.dock_batch_noalloc(pocket, gl, out, 256, 10, timeout_ns=1, stream=stream)
    torch.cuda.synchronize()
    res = out.cpu().numpy().view(dock.RESULT_DTYPE)
    np.testing.assert_array_equal(res["status"], dock.DOCK_ETIMEOUT)
    dock.dock_batch_noalloc(pocket, gl, out, 64, 2, stream=stream)
    torch.cuda.synchronize()
    res = out.cpu().numpy().view(dock.RESULT_DTYPE)
    np.testing.assert_array_equal(res["status"], 0)
