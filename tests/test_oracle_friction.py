"""Pins of the oracle's ground friction (Sec. 4.2, friction energy).

Friction adds k_f |v_h(x)|^2 ReLU(eps - y0) per vertex to the potential of a
backward-Euler step, with v(x) = (x - x0)/h and v_h its horizontal part (all
axes except y).  Checked here: derivatives against finite differences, the
closed-form backward-Euler update of independent particles with linear drag,
the impulse balance of a whole step, and the adjoint of a rollout against
finite differences in every input (activations, x0, v0).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth

K_F, EPS_F = 2e3, 0.01


def _problem(kind):
    if kind == "tri":
        p = synth.make_small2d(4, 2, fix_bottom=False)
    else:
        p = synth.make_small3d(2, 2, 2, split=5, fix_bottom=False)
    p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
    p.k_friction, p.eps_friction = K_F, EPS_F
    return p


@pytest.fixture(params=["tri", "tet5"])
def kind(request):
    return request.param


def _x0(p, rng):
    """Previous positions: rest shape lifted so that some vertices sit below eps."""
    x0 = p.X + 0.002 * rng.standard_normal(p.X.shape)
    x0[:, 1] += 0.004
    return x0


def test_friction_model_defaults_off():
    p = synth.make_small2d(4, 2)
    assert oracle.make_model(p).k_friction == 0.0


def test_friction_gradient_and_hvp_match_fd(kind):
    p = _problem(kind)
    rng = np.random.default_rng(31)
    x0 = _x0(p, rng)
    v0 = 0.3 * rng.standard_normal(x0.shape)
    m = oracle.make_model(p).replace(x0=x0, xhat=x0 + p.dt * v0)
    assert (x0[:, 1] < EPS_F).any() and (x0[:, 1] > EPS_F).any()
    x = x0 + 0.01 * rng.standard_normal(x0.shape)
    g = m.grad(x, p.a)
    dx = rng.standard_normal(x.shape)
    eps = 1e-6
    fd = (m.energy(x + eps * dx, p.a) - m.energy(x - eps * dx, p.a)) / (2 * eps)
    assert math.isclose(fd, float(np.sum(g * dx)), rel_tol=1e-6)
    Hv = m.hvp(x, p.a, dx)
    fdh = (m.grad(x + eps * dx, p.a) - m.grad(x - eps * dx, p.a)) / (2 * eps)
    assert np.abs(fdh - Hv).max() < 1e-6 * np.abs(Hv).max()
    # friction is really switched on in this model
    m0 = m.replace(k_friction=0.0)
    assert abs(m.energy(x, p.a) - m0.energy(x, p.a)) > 1e-3 * abs(m.energy(x, p.a) - m.energy(x0, p.a))


def test_friction_acts_only_below_eps_and_horizontally(kind):
    p = _problem(kind)
    rng = np.random.default_rng(32)
    x0 = _x0(p, rng)
    m = oracle.make_model(p).replace(x0=x0, xhat=x0.copy())
    m0 = m.replace(k_friction=0.0)
    # a purely vertical move costs no friction
    xv = x0.copy()
    xv[:, 1] += 0.003 * rng.standard_normal(len(x0))
    assert m.energy(xv, p.a) == m0.energy(xv, p.a)
    # nothing happens when every previous position is above eps
    up = x0.copy()
    up[:, 1] += 1.0
    mu = m.replace(x0=up, xhat=up.copy())
    x = up + 0.01 * rng.standard_normal(up.shape)
    assert mu.energy(x, p.a) == mu.replace(k_friction=0.0).energy(x, p.a)
    # quasistatic models never see friction
    mq = m.replace(h=0.0, xhat=None)
    assert mq.energy(x0 + 0.01, p.a) == mq.replace(k_friction=0.0).energy(x0 + 0.01, p.a)


def test_drag_on_free_particles_matches_backward_euler_closed_form(kind):
    """With no elasticity, gravity or contact every vertex is a particle under
    linear drag; backward Euler gives v1 = m v0 / (m + 2 k_f ReLU(eps - y0))
    on the horizontal axes and leaves y alone."""
    p = _problem(kind)
    rng = np.random.default_rng(33)
    x0 = _x0(p, rng)
    m = oracle.make_model(p).replace(mu=0.0, lam=0.0, k_muscle=0.0, gravity=0.0, k_contact=0.0)
    v0 = np.zeros_like(x0)
    v0[:, 0] = 0.05 * (1.0 + rng.uniform(size=len(x0)))
    if p.dim == 3:
        v0[:, 2] = -0.04 * (1.0 + rng.uniform(size=len(x0)))
    x1, v1, st = oracle.be_step(m, x0, v0, p.a, rtol=1e-13)
    assert st["status"] == oracle.OK
    damp = m.mass / (m.mass + 2.0 * K_F * np.maximum(EPS_F - x0[:, 1], 0.0))
    for c in range(p.dim):
        want = v0[:, c] * (1.0 if c == 1 else damp)
        assert np.abs(v1[:, c] - want).max() < 1e-9 * np.abs(v0).max()
    assert (damp < 0.9).any() and (damp == 1.0).any()


def test_step_impulse_balance(kind):
    """Internal forces sum to zero, so over one step the horizontal momentum
    changes by the friction impulse alone, and y by gravity and contact alone."""
    p = _problem(kind)
    rng = np.random.default_rng(34)
    x0 = _x0(p, rng)
    v0 = 0.2 * rng.standard_normal(x0.shape)
    m = oracle.make_model(p)
    x1, v1, st = oracle.be_step(m, x0, v0, p.a, rtol=1e-13)
    assert st["status"] == oracle.OK
    dP = (m.mass[:, None] * (v1 - v0)).sum(axis=0)
    fw = 2.0 * K_F * np.maximum(EPS_F - x0[:, 1], 0.0)
    scale = np.abs(m.mass[:, None] * v0).sum()
    for c in range(p.dim):
        if c == 1:
            continue
        assert abs(dP[c] + np.sum(fw * v1[:, c])) < 1e-9 * scale
        assert abs(np.sum(fw * v1[:, c])) > 1e-3 * scale
    # vertical: m dv_y = -h (m g + dC/dy(y1)) summed; friction adds nothing
    mq = m.replace(h=0.0, mu=0.0, lam=0.0, k_muscle=0.0, k_friction=0.0)
    fy = mq.grad(x1, np.zeros(p.n_elem))[:, 1].sum()
    assert abs(dP[1] + m.h * fy) < 1e-9 * (scale + m.h * abs(fy))


def test_rollout_adjoint_with_friction_matches_fd(kind):
    p = _problem(kind)
    m = oracle.make_model(p)
    rng = np.random.default_rng(35)
    nT = 3
    a_seq = rng.uniform(0.0, 1.0, size=(nT, p.n_elem))
    x0 = _x0(p, rng)
    v0 = 0.2 * rng.standard_normal(x0.shape)
    xs, vs = oracle.rollout(m, x0, v0, a_seq, rtol=1e-13)
    # every step has vertices both in and out of the friction band, away from the kink
    for x in xs[:-1]:
        assert (x[:, 1] < EPS_F).any() and np.abs(x[:, 1] - EPS_F).min() > 1e-4
    c = rng.standard_normal(x0.shape)
    cv = 0.01 * rng.standard_normal(x0.shape)

    def loss(xT, vT):
        return float(np.sum(c * xT) + np.sum(cv * vT))

    xbar0, vbar0, abar = oracle.rollout_backward(m, xs, vs, a_seq, c, cv)
    eps = 1e-6
    for what, d in (("a", rng.standard_normal(a_seq.shape)), ("x0", rng.standard_normal(x0.shape)),
                    ("v0", rng.standard_normal(x0.shape))):
        args_p = [x0, v0, a_seq]
        args_m = [x0, v0, a_seq]
        i = {"x0": 0, "v0": 1, "a": 2}[what]
        args_p[i] = args_p[i] + eps * d
        args_m[i] = args_m[i] - eps * d
        xp, vp = oracle.rollout(m, *args_p, rtol=1e-13)
        xm, vm = oracle.rollout(m, *args_m, rtol=1e-13)
        fd = (loss(xp[-1], vp[-1]) - loss(xm[-1], vm[-1])) / (2 * eps)
        an = float(np.sum({"a": abar, "x0": xbar0, "v0": vbar0}[what] * d))
        assert math.isclose(fd, an, rel_tol=2e-5), what
    # friction matters to the gradient
    m0 = m.replace(k_friction=0.0)
    xs0, vs0 = oracle.rollout(m0, x0, v0, a_seq, rtol=1e-13)
    _, _, abar0 = oracle.rollout_backward(m0, xs0, vs0, a_seq, c, cv)
    assert np.abs(abar - abar0).max() > 1e-3 * np.abs(abar).max()
