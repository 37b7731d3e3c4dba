"""The C-ABI library loads and exports every entry point that include/hz.h declares
(no compute calls: runs without a GPU)."""
import os
import re

from paper_1801_08655_gb300 import build, hz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "hz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hz_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    path = build.build()
    names = declared()
    assert len(names) >= 16
    import ctypes
    lib = ctypes.CDLL(path)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(hz.exported_symbols(path)) == sorted(set(hz.EXPORTED))
    assert set(hz.EXPORTED) == set(names)


def test_default_options():
    o = hz.default_opts("fp64")
    assert o.gmres_tol == 1e-10 and o.restart == 12
    o = hz.default_opts("mixed")
    assert o.gmres_tol == 1e-7 and o.max_refine == 3 and o.krylov == 0


def test_binding_refuses_to_run_without_library(tmp_path):
    import pytest
    with pytest.raises(ImportError):
        hz._lib_saved = hz._lib
        hz._lib = None
        try:
            hz.load(str(tmp_path / "missing.so"))
        finally:
            hz._lib = hz._lib_saved
