"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/softsim.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "softsim.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(sim_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2102_05791_gb300.build import build
    return build()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("sim_create", "sim_destroy", "sim_energy_grad", "sim_hvp", "sim_newton_solve",
                 "sim_adjoint_solve", "sim_param_vjp"):
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    from paper_2102_05791_gb300 import _lib
    assert sorted(_lib.EXPORTED) == _declared()
    _lib.load(lib_path)


def test_default_options_on_host(lib_path):
    from paper_2102_05791_gb300 import _lib
    L = _lib.load(lib_path)
    o = _lib.SimOptions()
    assert L.sim_default_options(ctypes.byref(o)) == 0
    assert o.precision == _lib.SIM_PREC_MIXED and o.newton_rtol == 1e-8 and o.max_cg == 500
    assert L.sim_default_options(None) == _lib.SIM_EINVAL


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror has the C struct's size and field offsets (gcc on the header)."""
    import subprocess

    from paper_2102_05791_gb300 import _lib
    structs = {"sim_mesh": _lib.SimMesh, "sim_material": _lib.SimMaterial, "sim_options": _lib.SimOptions,
               "sim_solve_stats": _lib.SimStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "softsim.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {cf}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln)}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
