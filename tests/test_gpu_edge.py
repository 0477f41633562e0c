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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_all_options_together_step_and_backward(precision):
    """Tet mesh with the quadratic log, the spring muscle, ground friction and
    the paper's quadratic contact: one backward-Euler step, its backward and
    the material VJPs at the step's adjoint, against the oracle."""
    import oracle
    p = synth.make_small3d(3, 2, 3, split=6, fix_bottom=False, seed=120)
    p.k_contact, p.contact_power, p.dt = 1e5, 2, 1.0 / 30.0
    p.k_friction, p.eps_friction = 2e3, 0.01
    p.log_mode, p.muscle_model = 1, 1
    p.a = 0.5 + 0.5 * p.a
    sim = make_sim(p, precision, tile_elems=16, k_friction=p.k_friction, eps_friction=p.eps_friction,
                   muscle_model=1, adjoint_rtol=1e-10 if precision == "fp64" else 1e-7)
    m = oracle.make_model(p)
    rng = np.random.default_rng(121)
    x0 = p.X + 0.002 * rng.standard_normal(p.X.shape)
    x0[:, 1] += 0.004
    v0 = 0.3 * rng.standard_normal(x0.shape)
    x1, v1, st = sim.step(dev(x0), dev(v0), dev(p.a))
    assert st["status"] == 0, st
    x1_or, _, _ = oracle.be_step(m, x0, v0, p.a, rtol=1e-10)
    assert np.abs(host(x1) - x1_or).max() <= 1e-5 * np.abs(x1_or - x0).max()
    xb1 = rng.standard_normal(x0.shape)
    vb1 = rng.standard_normal(x0.shape)
    xb0, vb0, ab, _ = sim.step_backward(dev(x0), dev(v0), x1, dev(p.a), dev(xb1), dev(vb1))
    xb0_or, vb0_or, ab_or = oracle.be_step_backward(m, x0, v0, host(x1), p.a, xb1, vb1)
    tol = 1e-7 if precision == "fp64" else 1e-4
    for got, ref in ((xb0, xb0_or), (vb0, vb0_or), (ab, ab_or)):
        assert np.linalg.norm(host(got) - ref) <= tol * np.linalg.norm(ref)
    # material VJPs at the oracle's adjoint of this step (backward-Euler scaling)
    ms = m.replace(xhat=x0 + p.dt * v0, x0=x0)
    lam, _ = ms.adjoint(host(x1), p.a, xb1 + vb1 / p.dt)
    got = sim.material_vjp(x1, dev(p.a), dev(lam))
    for g, r in zip(got, ms.material_vjp(host(x1), lam, p.a)):
        assert np.abs(host(g) - r).max() <= 1e-12 * np.abs(r).max()


def test_batch_quadratic_log():
    from paper_2102_05791_gb300.api import Batch
    import oracle
    probs = []
    for i, (nx, ny) in enumerate([(4, 2), (5, 3)]):
        p = synth.make_small2d(nx, ny, fix_bottom=False, seed=130 + i)
        p.k_contact, p.contact_power, p.dt, p.log_mode = 1e6, 3, 1.0 / 30.0, 1
        probs.append(p)
    b = Batch(probs, adjoint_rtol=1e-8)
    rng = np.random.default_rng(131)
    a_seq = rng.uniform(0.0, 1.0, size=(3, b.E))
    x0 = np.concatenate([p.X for p in probs])
    v0 = 0.1 * rng.standard_normal(x0.shape)
    xbT = rng.standard_normal(x0.shape)
    sx, sv, abar, xb0, vb0, ms = b.rollout(dev(x0), dev(v0), dev(a_seq), dev(xbT), dev(np.zeros_like(x0)))
    torch.cuda.synchronize()
    assert (host(ms)[:, 0] == 0).all()
    sx, abar = host(sx), host(abar)
    vo, eo = b.vert_offsets, b.elem_offsets
    for i, p in enumerate(probs):
        m = oracle.make_model(p)
        assert m.log_mode == 1
        a_i = a_seq[:, eo[i]:eo[i + 1]]
        xs, vs = oracle.rollout(m, x0[vo[i]:vo[i + 1]], v0[vo[i]:vo[i + 1]], a_i, rtol=1e-10)
        assert np.abs(sx[-1, vo[i]:vo[i + 1]] - xs[-1]).max() <= 1e-6 * np.abs(xs[-1] - xs[0]).max()
        _, _, ab = oracle.rollout_backward(m, xs, vs, a_i, xbT[vo[i]:vo[i + 1]], np.zeros_like(p.X))
        assert np.linalg.norm(abar[:, eo[i]:eo[i + 1]] - ab) <= 1e-4 * np.linalg.norm(ab)
    b.close()
