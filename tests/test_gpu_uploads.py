"""dock_batch's host tables (genotype offsets, work items, Solis-Wets units)
reach the device three ways: copied on the workspace's own stream into
buffers a call has just allocated, copied on the caller's stream when they
changed in buffers earlier searches may still read, or not copied when the
device already holds them. Whatever sequence of settings one ligand set sees,
every search must give the records a fresh ligand set gives for the same
settings; and searches queued back to back on one stream must each read their
own records."""
import numpy as np
import pytest

from helpers import gpu_ligands, gpu_pocket
from paper_2509_12232_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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
def setup(dock):
    pk, _, _ = synth.make_workload("c1")
    rng = np.random.Generator(np.random.Philox(5150))
    ligs = synth.make_ligands(rng, np.array([12, 25, 50, 90, 3, 40]), np.array([2, 5, 9, 16, 0, 6]),
                              id_base=300)
    pocket = gpu_pocket(dock, pk)
    return dict(pk=pk, ligs=ligs, pocket=pocket)


def _records(dock, pocket, gl, pop, gens, **kw):
    job = dock.dock_batch(pocket, gl, pop, gens, seed=4, stream=torch.cuda.current_stream(),
                          **SEARCH, **kw)
    r = dock.dock_results(job)
    job.close()
    return r


def _same(a, b, what):
    for name in a.dtype.names:
        np.testing.assert_array_equal(a[name], b[name], err_msg="%s: %s" % (what, name))


def test_settings_changing_on_one_ligand_set(dock, setup):
    pocket, ligs = setup["pocket"], setup["ligs"]
    ls = dock.ls_params(0.1, 20)
    runs = [dict(pop=64, gens=3), dict(pop=32, gens=3), dict(pop=64, gens=3),
            dict(pop=64, gens=3, ls=ls), dict(pop=96, gens=2, ls=ls), dict(pop=64, gens=3),
            dict(pop=64, gens=3, lanes_per_pose=8), dict(pop=64, gens=3)]
    gl = gpu_ligands(dock, pocket, ligs)
    for i, kw in enumerate(runs):
        kw = dict(kw)
        pop, gens = kw.pop("pop"), kw.pop("gens")
        got = _records(dock, pocket, gl, pop, gens, **kw)
        fresh = gpu_ligands(dock, pocket, ligs)
        ref = _records(dock, pocket, fresh, pop, gens, **kw)
        fresh.close()
        assert np.all(got["status"] == 0)
        _same(got, ref, "run %d" % i)
    gl.close()


def test_searches_queued_back_to_back(dock, setup):
    """Three searches on three ligand sets queued on one stream before any
    result is read: each job's records are its own."""
    pocket, ligs = setup["pocket"], setup["ligs"]
    refs = []
    for pop in (32, 64, 48):
        g = gpu_ligands(dock, pocket, ligs)
        refs.append(_records(dock, pocket, g, pop, 3))
        g.close()
    sets = [gpu_ligands(dock, pocket, ligs) for _ in range(3)]
    jobs = [dock.dock_batch(pocket, g, pop, 3, seed=4, stream=torch.cuda.current_stream(), **SEARCH)
            for g, pop in zip(sets, (32, 64, 48))]
    for j, ref in zip(jobs, refs):
        _same(dock.dock_results(j), ref, "queued")
        j.close()
    for g in sets:
        g.close()
