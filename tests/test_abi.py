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


def test_ctypes_mirrors_match_the_c_struct_layouts(tmp_path):
    """Every struct that the binding mirrors has the size and field offsets that a C compiler
    gives the declarations in include/hz.h (compiled here with gcc; no GPU)."""
    import ctypes
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"hz_grid": hz.Grid, "hz_pml": hz.Pml, "hz_solve_opts": hz.SolveOpts, "hz_solve_info": hz.SolveInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hz.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
