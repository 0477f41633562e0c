"""sim_energy_noalloc: the energy of a mesh held in caller-owned device arrays,
evaluated without allocating device memory.

Callers whose GPU memory is already claimed by another framework's pool, or
that must not allocate after setup, use this entry point instead of a handle.
It is checked here against the handle-based sim_energy_grad and against the
FP64 oracle's energy on two calls in a row, the second of which reuses the
scratch array the first one left behind; the device's free memory must not
change across those calls.  A rest mesh with an inverted element is reported
as SIM_EINVERTED.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
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


def _call(L, p, X, T, x, a, fiber, mat, E):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.sim_energy_noalloc(p.dim, p.n_vert, p.n_elem, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                C.c_void_p(x.data_ptr()), C.c_void_p(a.data_ptr()), C.c_void_p(fiber.data_ptr()),
                                C.byref(mat), C.c_void_p(E.data_ptr()), stream)


@pytest.mark.parametrize("muscle", [0, 1], ids=["contractile", "spring"])
@pytest.mark.parametrize("name", ["c1", "small3d"])
def test_energy_noalloc_matches_handle_and_oracle_twice(name, muscle):
    from paper_2102_05791_gb300 import _lib
    L = _lib.load()
    p = synth.make_config1() if name == "c1" else synth.make_small3d(6, 4, 4, split=6, seed=51)
    p.k_contact = 1e5
    p.muscle_model = muscle
    if muscle:
        p.a = 0.5 + 0.5 * p.a  # the spring needs a > 0
    sim = make_sim(p, "fp64", muscle_model=muscle)
    m = oracle.make_model(p)
    mat = _material(p)
    X, T = dev(p.X), torch.from_numpy(p.T).cuda().contiguous()
    fiber, a = dev(p.fiber), dev(p.a)
    states = []
    for call in range(2):
        x = deformed(p, 0.03, seed=1 + call)
        x[:, 1] -= 0.01 * call  # second call: some vertices below ground, contact term active
        states.append((x, dev(x)))
    E = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    # warm-up: the first call loads the kernel and looks up the scratch address
    assert _call(L, p, X, T, states[0][1], a, fiber, mat, E) == 0, L.sim_noalloc_last_error().decode()
    E_ref = [float(sim.energy_grad(xd, a)[0]) for _, xd in states]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    got = []
    for _, xd in states:
        E.fill_(float("nan"))
        rc = _call(L, p, X, T, xd, a, fiber, mat, E)
        assert rc == 0, L.sim_noalloc_last_error().decode()
        got.append(float(E))
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)  # nothing allocated on the device
    for call, ((x, _), Eg, Eh) in enumerate(zip(states, got, E_ref)):
        assert abs(Eg - Eh) <= TOL64 * max(abs(Eh), 1.0), (call, Eg, Eh)
        E_or, S_or = m.energy(x, p.a, with_abs=True)
        assert abs(Eg - E_or) <= TOL64 * S_or, (call, Eg, E_or)
    sim.close()


def test_energy_noalloc_reports_an_inverted_rest_element():
    from paper_2102_05791_gb300 import _lib
    L = _lib.load()
    p = synth.make_small2d(4, 2)
    T = p.T.copy()
    T[3, [1, 2]] = T[3, [2, 1]]  # one triangle with negative rest area
    mat = _material(p)
    E = torch.zeros((), dtype=torch.float64, device="cuda")
    rc = _call(L, p, dev(p.X), torch.from_numpy(T).cuda().contiguous(), dev(p.X), dev(p.a), dev(p.fiber), mat, E)
    assert rc == _lib.SIM_EINVERTED
    assert b"non-positive" in L.sim_noalloc_last_error()
    assert np.isnan(float(E))


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
