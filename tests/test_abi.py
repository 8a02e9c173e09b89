"""CPU checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/dock.h declares; the binding refuses to run
without it (no fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dock.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(dock_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2509_12232_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("dock_create_pocket", "dock_load_ligands", "dock_batch", "dock_results", "dock_score",
              "dock_last_error", "dock_pocket_destroy", "dock_ligands_destroy", "dock_job_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_version(libpath):
    from paper_2509_12232_gb300 import dock
    assert "sm_103a" in dock.version()


def test_binding_raises_without_library(tmp_path, monkeypatch):
    from paper_2509_12232_gb300 import dock
    monkeypatch.setattr(dock, "_lib", None)
    monkeypatch.setattr(dock, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        dock.lib()


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler
    gives the header's structs."""
    import subprocess
    from paper_2509_12232_gb300 import dock
    structs = {
        "dock_type_params": dock.dock_type_params,
        "dock_pocket_desc": dock.dock_pocket_desc,
        "dock_ligand_batch": dock.dock_ligand_batch,
        "dock_search_params": dock.dock_search_params,
        "dock_ls_params": dock.dock_ls_params,
        "dock_result": dock.dock_result,
        "dock_train_params": dock.dock_train_params,
        "dock_tune_table": dock.dock_tune_table,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dock.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (name, f)]) == getattr(cls, f).offset, (name, f)
    assert ctypes.sizeof(dock.dock_result) == dock.RESULT_DTYPE.itemsize
