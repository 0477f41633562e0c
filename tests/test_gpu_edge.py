"""Degenerate inputs on the GPU: a start already at equilibrium, a zero
adjoint right-hand side, a mesh with every vertex pinned, and zero-step
rollouts.  Each has an exact answer (no iterations, zeros, identities)."""
import numpy as np
import pytest
import torch

import synth
from simhelp import dev, host, make_sim

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["tri", "tet"])
def test_equilibrium_start_and_zero_rhs(kind, precision):
    """a = 0 and no gravity: the rest shape is the minimiser (E = 0, grad = 0),
    the solve takes no Newton step, and a zero dL/dx gives lambda = 0."""
    p = synth.make_small2d(6, 3) if kind == "tri" else synth.make_small3d(3, 2, 2, split=5)
    p.gravity = 0.0
    a = dev(np.zeros(p.n_elem))
    sim = make_sim(p, precision, tile_elems=16)
    E, g = sim.energy_grad(dev(p.X), a)
    assert float(E) == 0.0 and float(torch.abs(g).max()) == 0.0
    x, st = sim.solve(a)
    assert st["status"] == 0 and st["newton_iters"] == 0
    assert torch.equal(x, dev(p.X))
    lam, sta = sim.adjoint(x, a, torch.zeros_like(x))
    assert sta["status"] == 0 and sta["cg_iters_total"] == 0
    assert float(torch.abs(lam).max()) == 0.0


def test_all_vertices_pinned():
    """Every vertex pinned: gradient and HVP vanish, the solve returns the
    rest shape and the adjoint is zero whatever dL/dx is."""
    p = synth.make_small2d(4, 2)
    p.fixed[:] = 1
    sim = make_sim(p, "mixed", tile_elems=16)
    a = dev(p.a)
    x = dev(p.X + 0.01)
    _, g = sim.energy_grad(x, a)
    assert float(torch.abs(g).max()) == 0.0
    Hv = sim.hvp(x, a, dev(np.ones(p.X.shape), sim.vec_dtype))
    assert float(torch.abs(Hv).max()) == 0.0
    xs, st = sim.solve(a)
    assert st["status"] == 0 and torch.equal(xs, dev(p.X))
    lam, _ = sim.adjoint(xs, a, torch.ones_like(xs))
    assert float(torch.abs(lam).max()) == 0.0


def test_zero_step_rollout_is_the_identity():
    p = synth.make_small2d(4, 2, fix_bottom=False)
    p.k_contact, p.dt = 1e6, 1.0 / 30.0
    sim = make_sim(p, "mixed", tile_elems=16)
    x0 = dev(p.X)
    v0 = dev(0.1 * np.random.default_rng(1).standard_normal(p.X.shape))
    a_seq = dev(np.zeros((0, p.n_elem)))
    xT, vT, ck, st = sim.rollout(x0, v0, a_seq, ckpt_every=5)
    assert torch.equal(xT, x0) and torch.equal(vT, v0)
    xb = dev(np.random.default_rng(2).standard_normal(p.X.shape))
    vb = dev(np.random.default_rng(3).standard_normal(p.X.shape))
    xb0, vb0, ab, _ = sim.rollout_backward(a_seq, ck, 5, xb, vb)
    assert torch.equal(xb0, xb) and torch.equal(vb0, vb) and ab.numel() == 0
