"""sim_energy_noalloc: the energy of a mesh held in caller-owned device arrays,
evaluated without allocating device memory.

Callers whose GPU memory is already claimed by another framework's pool, or
that must not allocate after setup, use this entry point instead of a handle.
It is checked here against the handle-based sim_energy_grad on two calls in a
row, the second of which reuses the scratch array the first one left behind.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from simhelp import deformed, dev, make_sim

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _material(p):
    from paper_2102_05791_gb300 import _lib
    mat = _lib.SimMaterial(p.mu, p.lam, p.k_muscle, p.density, p.gravity, p.k_contact, p.contact_power,
                           p.log_mode, 0.0, None)
    mat.muscle_model = p.muscle_model
    return mat


@pytest.mark.parametrize("muscle", [0, 1], ids=["contractile", "spring"])
@pytest.mark.parametrize("name", ["c1", "small3d"])
def test_energy_noalloc_matches_handle_energy_twice(name, muscle):
    from paper_2102_05791_gb300 import _lib
    L = _lib.load()
    p = synth.make_config1() if name == "c1" else synth.make_small3d(6, 4, 4, split=6, seed=51)
    p.k_contact = 1e5
    p.muscle_model = muscle
    if muscle:
        p.a = 0.5 + 0.5 * p.a  # the spring needs a > 0
    sim = make_sim(p, "fp64", muscle_model=muscle)
    mat = _material(p)
    X, T = dev(p.X), torch.from_numpy(p.T).cuda().contiguous()
    fiber, a = dev(p.fiber), dev(p.a)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((1, 2)):
        x = deformed(p, 0.03, seed=seed)
        x[:, 1] -= 0.01 * call  # second call: some vertices below ground, contact term active
        xd = dev(x)
        E_ref, _ = sim.energy_grad(xd, a)
        E = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.sim_energy_noalloc(p.dim, p.n_vert, p.n_elem, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                  C.c_void_p(xd.data_ptr()), C.c_void_p(a.data_ptr()),
                                  C.c_void_p(fiber.data_ptr()), C.byref(mat), C.c_void_p(E.data_ptr()), stream)
        assert rc == 0, L.sim_noalloc_last_error().decode()
        torch.cuda.synchronize()
        assert abs(float(E) - float(E_ref)) <= TOL64 * max(abs(float(E_ref)), 1.0), (call, float(E), float(E_ref))
    sim.close()


def test_energy_noalloc_rejects_oversized_mesh():
    from paper_2102_05791_gb300 import _lib
    L = _lib.load()
    p = synth.make_small2d(2, 1)
    mat = _material(p)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    ptr = C.c_void_p(buf.data_ptr())
    rc = L.sim_energy_noalloc(2, 5_000_000, 5_000_000, ptr, ptr, ptr, ptr, ptr, C.byref(mat), ptr, None)
    assert rc == _lib.SIM_EINVAL
    assert b"too large" in L.sim_noalloc_last_error()
