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


def _valid_inputs():
    import numpy as np

    from paper_2102_05791_gb300 import _lib
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    T = np.array([[0, 1, 2]], dtype=np.int32)
    fib = np.array([[1.0, 0.0]])
    keep = (X, T, fib)
    mesh = _lib.SimMesh(2, 3, 1, X.ctypes.data, T.ctypes.data, None)
    mat = _lib.SimMaterial(1e4, 4e4, 5e3, 1e3, 9.8, 0.0, 3, 0, 0.0, fib.ctypes.data, 0.0, 0.01, 0)
    return keep, mesh, mat


@pytest.mark.parametrize("case,msg", [
    ("dim", b"dim must be 2 or 3"),
    ("empty", b"empty mesh"),
    ("huge", b"too large"),
    ("cpow", b"contact_power"),
    ("log", b"log_mode"),
    ("muscle", b"muscle_model"),
    ("dt", b"bad material scalar"),
    ("nan_mu", b"bad material scalar"),
    ("friction", b"k_friction"),
    ("precision", b"precision"),
])
def test_create_rejects_invalid_inputs_before_touching_the_gpu(lib_path, case, msg):
    """sim_create validates its host arguments first: each bad input returns
    SIM_EINVAL with a message (no GPU call is made, so this runs on the CPU)."""
    from paper_2102_05791_gb300 import _lib
    L = _lib.load(lib_path)
    keep, mesh, mat = _valid_inputs()
    opt = _lib.SimOptions()
    L.sim_default_options(ctypes.byref(opt))
    if case == "dim":
        mesh.dim = 4
    elif case == "empty":
        mesh.n_elem = 0
    elif case == "huge":
        mesh.n_vert = (1 << 30) + 1
    elif case == "cpow":
        mat.contact_power = 4
    elif case == "log":
        mat.log_mode = 7
    elif case == "muscle":
        mat.muscle_model = 2
    elif case == "dt":
        mat.dt = -1.0
    elif case == "nan_mu":
        mat.mu = float("nan")
    elif case == "friction":
        mat.k_friction = -1.0
    elif case == "precision":
        opt.precision = 5
    h = ctypes.c_void_p()
    rc = L.sim_create(ctypes.byref(mesh), ctypes.byref(mat), ctypes.byref(opt), ctypes.byref(h))
    assert rc == _lib.SIM_EINVAL
    assert not h.value
    assert msg in L.sim_last_error(None)
    assert L.sim_create(None, ctypes.byref(mat), ctypes.byref(opt), ctypes.byref(h)) == _lib.SIM_EINVAL
