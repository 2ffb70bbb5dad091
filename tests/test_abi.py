"""The C-ABI library builds for sm_103a, loads, and exports every function include/dg.h declares."""
import ctypes
import os
import subprocess

import pytest

from paper_2306_01085_gb300 import build as B
from paper_2306_01085_gb300 import dg as DG
from paper_2306_01085_gb300 import workloads as W


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    names = DG.declared_functions()
    assert "dg_residual" in names and "dg_jvp" in names and "dg_mesh_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("cname,pytype", [("dg_mesh_desc", DG.DgMeshDesc), ("dg_solver_opts", DG.DgSolverOpts),
                                          ("dg_step_stats", DG.DgStepStats)])
def test_struct_layouts_match_header(tmp_path, cname, pytype):
    """ctypes mirrors of the ABI structs have the C layout (size and every field offset)."""
    fields = [f for f, _ in pytype._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.abspath(DG.HEADER)}"',
             "int main(void) {", f'printf("%zu\\n", sizeof({cname}));']
    lines += [f'printf("%zu\\n", offsetof({cname}, {f}));' for f in fields]
    lines += ["return 0; }"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(pytype)
    for f, off in zip(fields, out[1:]):
        assert getattr(pytype, f).offset == off, f


def test_descriptor_roundtrip():
    d = W.shell_desc(n=4, nr=2, p=3, euv=True)
    c = DG.to_c_desc(d)
    assert c.p == 3 and c.nx == 4 and abs(c.grashof - d.grashof) < 1e-9 * d.grashof
    assert list(c.omega) == list(d.omega) and c.euv == 1
    d2 = W.shell_desc(n=2, nr=2, p=1, euvac=True, composition=True)
    c2 = DG.to_c_desc(d2)
    assert c2.euv == 2 and c2.comp == 1 and list(c2.comp_b) == list(d2.comp_b) and c2.ref_T0 == d2.ref_T0
