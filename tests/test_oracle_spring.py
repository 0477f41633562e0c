"""Pins of the oracle's active-spring muscle (Eq. active-spring-potential).

The spring model replaces the contractile term by (k/2)(|F f|/a - 1)^2 per
element (integrated over the element), |F f| being the fiber's stretch l/l0
for a unit rest fiber f.  Checked here: closed forms on one element
(energy, force, stiffness along and across the fiber, the action VJP),
zero force where every fiber sits at its target length, derivatives against
finite differences on small meshes, and the adjoint gradient of a
quasistatic solve against finite differences through the solve.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth

K = 5.0e3


def _unit(d, act, mu=0.0, lam=0.0):
    X = np.vstack([np.zeros(d), np.eye(d)])
    T = np.arange(d + 1, dtype=np.int32)[None, :]
    fib = np.zeros((1, d))
    fib[0, 0] = 1.0
    p = synth.SynthProblem("unit", d, X, T, np.zeros(d + 1, np.uint8), fib, np.array([act]), np.zeros(d),
                           mu=mu, lam=lam, k_muscle=K, gravity=0.0)
    p.muscle_model = 1
    return p, oracle.make_model(p, with_fixed=False)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("s,act", [(1.0, 0.6), (0.8, 0.6), (1.3, 0.9), (0.5, 1.0)])
def test_single_element_closed_forms(d, s, act):
    """F = diag(s, 1[, 1]) with the fiber along x: psi = k/2 (s/a - 1)^2; the
    stretched vertex feels W k (s/a - 1)/a along x; its stiffness is W k/a^2
    along the fiber and W k (s/a - 1)/(a s) across it; dL/da for lambda = e_x
    at that vertex is -W k (1/a^2 - 2 s/a^3)."""
    p, m = _unit(d, act)
    x = p.X.copy()
    x[1, 0] = s
    W = 1.0 / math.factorial(d)
    r = s / act - 1.0
    assert math.isclose(m.energy(x, p.a), W * 0.5 * K * r * r, rel_tol=1e-13, abs_tol=1e-12)
    g = m.grad(x, p.a)
    assert math.isclose(g[1, 0], W * K * r / act, rel_tol=1e-12, abs_tol=1e-9)
    assert abs(g[1, 1:]).max() < 1e-9 and np.abs(g.sum(axis=0)).max() < 1e-9
    v = np.zeros_like(x)
    v[1, 0] = 1.0
    Hv = m.hvp(x, p.a, v)
    assert math.isclose(Hv[1, 0], W * K / act ** 2, rel_tol=1e-12)
    v = np.zeros_like(x)
    v[1, 1] = 1.0
    Hv = m.hvp(x, p.a, v)
    assert math.isclose(Hv[1, 1], W * K * r / (act * s), rel_tol=1e-12, abs_tol=1e-9)
    lam = np.zeros_like(x)
    lam[1, 0] = 1.0
    vjp = m.param_vjp(x, lam, p.a)
    assert math.isclose(vjp[0], -W * K * (1.0 / act ** 2 - 2.0 * s / act ** 3), rel_tol=1e-12)


def test_fibers_at_target_length_feel_no_force():
    """Stretching a mesh by a along a common fiber direction puts every
    spring at its target length: zero muscle energy and force."""
    p = synth.make_small2d(4, 2)
    p.muscle_model = 1
    p.fiber[:] = [1.0, 0.0]
    act = 0.7
    a = np.full(p.n_elem, act)
    m = oracle.make_model(p, with_fixed=False).replace(mu=0.0, lam=0.0, gravity=0.0)
    x = p.X.copy()
    x[:, 0] *= act
    assert abs(m.energy(x, a)) < 1e-20
    assert np.abs(m.grad(x, a)).max() < 1e-10


def test_relaxed_spring_matches_contractile_curvature_at_rest():
    """At the rest shape with a = 1 the spring is at rest length: no force,
    and its stiffness along the fiber is k (the contractile term's k a with
    a = 1 has the same curvature along f, but a force k f)."""
    p, m = _unit(2, 1.0)
    x = p.X.copy()
    assert np.abs(m.grad(x, p.a)).max() < 1e-12
    v = np.zeros_like(x)
    v[1, 0] = 1.0
    mc = m.replace(muscle_model=0)
    assert math.isclose(m.hvp(x, p.a, v)[1, 0], mc.hvp(x, p.a, v)[1, 0], rel_tol=1e-13)
    assert math.isclose(mc.grad(x, p.a)[1, 0], 0.5 * K, rel_tol=1e-13)


def _spring_problem(kind):
    if kind == "tri":
        p = synth.make_small2d(4, 2)
    else:
        p = synth.make_small3d(2, 2, 2, split=5)
    p.muscle_model = 1
    p.a = 0.5 + 0.5 * p.a  # actions in [0.5, 1]
    return p


@pytest.fixture(params=["tri", "tet"])
def kind(request):
    return request.param


def test_spring_derivatives_match_fd(kind):
    p = _spring_problem(kind)
    rng = np.random.default_rng(21)
    m = oracle.make_model(p, with_fixed=False)
    x = p.X + 0.05 * rng.standard_normal(p.X.shape)
    u = rng.standard_normal(x.shape)
    eps = 1e-6
    fd = (m.energy(x + eps * u, p.a) - m.energy(x - eps * u, p.a)) / (2 * eps)
    assert math.isclose(fd, float(np.sum(m.grad(x, p.a) * u)), rel_tol=1e-7)
    Hu = m.hvp(x, p.a, u)
    fdh = (m.grad(x + eps * u, p.a) - m.grad(x - eps * u, p.a)) / (2 * eps)
    assert np.abs(fdh - Hu).max() < 1e-6 * np.abs(Hu).max()
    lam = rng.standard_normal(x.shape)
    vjp = m.param_vjp(x, lam, p.a)
    for e in range(0, p.n_elem, max(1, p.n_elem // 7)):
        da = np.zeros(p.n_elem)
        da[e] = 1e-5
        dg = (m.grad(x, p.a + da) - m.grad(x, p.a - da)) / 2e-5
        assert math.isclose(vjp[e], -np.sum(lam * dg), rel_tol=1e-6, abs_tol=1e-9 * np.abs(vjp).max())
    # the spring really differs from the contractile model here
    mc = m.replace(muscle_model=0)
    assert np.abs(mc.grad(x, p.a) - m.grad(x, p.a)).max() > 1e-2 * np.abs(m.grad(x, p.a)).max()


def test_spring_adjoint_gradient_matches_fd_through_solve(kind):
    p = _spring_problem(kind)
    m = oracle.make_model(p)
    x, lam, dLda, st = oracle.quasistatic_forward_backward(m, p.a, p.target, rtol=1e-12)
    assert st["status"] == oracle.OK
    rng = np.random.default_rng(22)
    delta = rng.standard_normal(p.n_elem)
    eps = 1e-5
    xp, _ = m.newton(p.a + eps * delta, rtol=1e-13)
    xm, _ = m.newton(p.a - eps * delta, rtol=1e-13)
    fd = (oracle.mean_loss(xp, p.target) - oracle.mean_loss(xm, p.target)) / (2 * eps)
    assert math.isclose(fd, float(dLda @ delta), rel_tol=1e-5)
