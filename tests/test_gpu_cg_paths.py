"""The two ways the library runs a CG solve agree.

SIM_CG_AUTO runs a whole CG solve of a mesh whose tiles fit on the GPU at
once as one kernel (tile data staged in shared memory once, two barriers per
iteration): as one thread-block cluster when the mesh has at most 16 tiles
(the small meshes here: cluster barrier, partial sums read from the other
CTAs' shared memory), else as a cooperative grid (the walker mesh in 32
tiles: L2 atomic barrier); SIM_CG_ITERATION launches the HVP tile kernel and
the small vector kernels per iteration.  Both solve the same systems with
different summation orders, so quasistatic solves, adjoints and a
backward-Euler step with its backward must agree within the parity
tolerances, and the cooperative path must launch far fewer kernels.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from simhelp import dev, host, make_sim

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["c1", "tet", "spring"])
def test_quasistatic_solve_and_adjoint_agree(kind, precision):
    if kind == "c1":
        p = synth.make_config1()
    else:
        p = synth.make_small3d(5, 3, 3, split=6 if kind == "tet" else 5, seed=71)
    kw = {}
    if kind == "spring":
        p.muscle_model = 1
        p.a = 0.5 + 0.5 * p.a
        kw["muscle_model"] = 1
    res = {}
    for mode in ("auto", "iteration"):
        sim = make_sim(p, precision, tile_elems=32, cg_kernel=mode, adjoint_rtol=1e-10, **kw)
        a = dev(p.a)
        n0 = sim.kernel_launches()
        x, st = sim.solve(a)
        assert st["status"] == 0, (mode, st)
        g = oracle.mean_loss_grad(host(x), p.target)
        lam, sta = sim.adjoint(x, a, dev(g))
        assert sta["status"] == 0, (mode, sta)
        res[mode] = (host(x), host(lam), sim.kernel_launches() - n0, st)
        sim.close()
    xa, la, na, sta_ = res["auto"]
    xi, li, ni, sti = res["iteration"]
    disp = np.abs(xi - p.X).max()
    assert np.abs(xa - xi).max() <= 1e-6 * disp
    assert np.linalg.norm(la - li) <= 1e-6 * np.linalg.norm(li)
    assert na < ni  # the cooperative kernel replaces the per-iteration launches


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dynamics_step_and_backward_agree(precision):
    p = synth.make_small2d(8, 4, fix_bottom=False, seed=73)
    p.k_contact, p.dt = 1e6, 1.0 / 30.0
    p.k_friction, p.eps_friction = 2e3, 0.01
    rng = np.random.default_rng(74)
    x0 = p.X + 0.002 * rng.standard_normal(p.X.shape)
    x0[:, 1] += 0.003
    v0 = 0.3 * rng.standard_normal(x0.shape)
    xb1, vb1 = rng.standard_normal(x0.shape), rng.standard_normal(x0.shape)
    out = {}
    for mode in ("auto", "iteration"):
        sim = make_sim(p, precision, tile_elems=16, cg_kernel=mode, adjoint_rtol=1e-10, k_friction=p.k_friction,
                       eps_friction=p.eps_friction)
        x1, v1, st = sim.step(dev(x0), dev(v0), dev(p.a))
        xb0, vb0, ab, _ = sim.step_backward(dev(x0), dev(v0), x1, dev(p.a), dev(xb1), dev(vb1))
        out[mode] = [host(t) for t in (x1, xb0, vb0, ab)]
        sim.close()
    x1a, *ga = out["auto"]
    x1i, *gi = out["iteration"]
    assert np.abs(x1a - x1i).max() <= 1e-6 * np.abs(x1i - x0).max()
    for a_, i_ in zip(ga, gi):
        assert np.linalg.norm(a_ - i_) <= 1e-6 * np.linalg.norm(i_)


def test_cooperative_path_matches_oracle_on_the_walker_mesh():
    """The 64 x 32 walker (32 tiles of 128 triangles, all resident), one
    backward-Euler step and its backward against the oracle."""
    p = synth.make_config2(n_steps=1)
    sim = make_sim(p, "mixed", tile_elems=128, adjoint_rtol=1e-10)
    x0, v0 = p.X.copy(), np.zeros_like(p.X)
    x1, v1, st = sim.step(dev(x0), dev(v0), dev(p.a))
    m = oracle.make_model(p)
    x1_or, _, _ = oracle.be_step(m, x0, v0, p.a, rtol=1e-10)
    assert np.abs(host(x1) - x1_or).max() <= 1e-5 * np.abs(x1_or - x0).max()
    xb1 = np.zeros_like(x0)
    xb1[:, 0] = 1.0 / p.n_vert
    xb0, vb0, ab, _ = sim.step_backward(dev(x0), dev(v0), x1, dev(p.a), dev(xb1), dev(np.zeros_like(x0)))
    _, _, ab_or = oracle.be_step_backward(m, x0, v0, host(x1), p.a, xb1, np.zeros_like(x0))
    assert np.linalg.norm(host(ab) - ab_or) <= 1e-4 * np.linalg.norm(ab_or)
    sim.close()
