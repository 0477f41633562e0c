"""Pins of the oracle's material-parameter VJPs: per-element dL/dmu,
dL/dlambda and dL/dk = -s lambda^T d(grad E)/dtheta_e (Eq. dLda-re-ordered
with a material parameter in place of the action).

Checked: closed forms on one stretched element; the sum over elements
against finite differences of the gradient in the global parameter (both
log modes, both muscle models, 2D and 3D); the adjoint gradient of a
quasistatic solve and of a backward-Euler step against finite differences
through the solve."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth

MU, LAM, K = 1.0e4, 4.0e4, 5.0e3


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("muscle", [0, 1])
@pytest.mark.parametrize("s", [0.7, 1.2])
def test_single_element_closed_forms(d, muscle, s):
    """F = diag(s, 1[, 1]), fiber along x, lambda = e_x on the stretched
    vertex: dL/dmu = -W (s - 1/s), dL/dlambda = -W log(s)/s, and dL/dk =
    -W a s (contractile) or -W (s/a - 1)/a (spring)."""
    act = 0.8
    X = np.vstack([np.zeros(d), np.eye(d)])
    T = np.arange(d + 1, dtype=np.int32)[None, :]
    fib = np.zeros((1, d))
    fib[0, 0] = 1.0
    p = synth.SynthProblem("unit", d, X, T, np.zeros(d + 1, np.uint8), fib, np.array([act]), np.zeros(d),
                           mu=MU, lam=LAM, k_muscle=K, gravity=0.0)
    p.muscle_model = muscle
    m = oracle.make_model(p, with_fixed=False)
    x = X.copy()
    x[1, 0] = s
    lam = np.zeros_like(x)
    lam[1, 0] = 1.0
    dmu, dlam, dk = m.material_vjp(x, lam, p.a)
    W = 1.0 / math.factorial(d)
    assert math.isclose(dmu[0], -W * (s - 1.0 / s), rel_tol=1e-12)
    assert math.isclose(dlam[0], -W * math.log(s) / s, rel_tol=1e-12)
    want_k = -W * act * s if muscle == 0 else -W * (s / act - 1.0) / act
    assert math.isclose(dk[0], want_k, rel_tol=1e-12)


def _prob(kind, muscle):
    p = synth.make_small2d(4, 2) if kind == "tri" else synth.make_small3d(2, 2, 2, split=5)
    p.muscle_model = muscle
    if muscle:
        p.a = 0.5 + 0.5 * p.a
    return p


@pytest.mark.parametrize("kind", ["tri", "tet"])
@pytest.mark.parametrize("log_mode", [0, 1])
@pytest.mark.parametrize("muscle", [0, 1])
def test_element_sums_match_fd_of_the_gradient(kind, log_mode, muscle):
    p = _prob(kind, muscle)
    rng = np.random.default_rng(61)
    m = oracle.make_model(p, log_mode=log_mode, with_fixed=False)
    x = p.X + 0.05 * rng.standard_normal(p.X.shape)
    lam = rng.standard_normal(x.shape)
    vjps = m.material_vjp(x, lam, p.a)
    for name, v in zip(("mu", "lam", "k_muscle"), vjps):
        th = getattr(m, name)
        eps = 1e-6 * th
        gp = m.replace(**{name: th + eps}).grad(x, p.a)
        gm = m.replace(**{name: th - eps}).grad(x, p.a)
        fd = -np.sum(lam * (gp - gm)) / (2 * eps)
        assert math.isclose(v.sum(), fd, rel_tol=1e-7, abs_tol=1e-9 * np.abs(v).sum()), name


@pytest.mark.parametrize("kind", ["tri", "tet"])
def test_quasistatic_material_gradient_matches_fd_through_solve(kind):
    p = _prob(kind, 0)
    m = oracle.make_model(p)
    x, lam, dLda, st = oracle.quasistatic_forward_backward(m, p.a, p.target, rtol=1e-12)
    assert st["status"] == oracle.OK
    dmu, dlam, dk = m.material_vjp(x, lam, p.a)
    for name, v in (("mu", dmu), ("lam", dlam), ("k_muscle", dk)):
        th = getattr(m, name)
        eps = 1e-5 * th
        xp, _ = m.replace(**{name: th + eps}).newton(p.a, rtol=1e-13)
        xm, _ = m.replace(**{name: th - eps}).newton(p.a, rtol=1e-13)
        fd = (oracle.mean_loss(xp, p.target) - oracle.mean_loss(xm, p.target)) / (2 * eps)
        assert math.isclose(fd, v.sum(), rel_tol=1e-5), name


def test_be_step_material_gradient_matches_fd():
    """One backward-Euler step: dL/dtheta = -h^2 lambda^T d(grad E)/dtheta
    with lambda = (M + h^2 H)^-1 dL/dx1."""
    p = synth.make_small2d(4, 2, fix_bottom=False)
    p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
    m = oracle.make_model(p)
    rng = np.random.default_rng(62)
    x0 = p.X.copy()
    v0 = 0.3 * rng.standard_normal(x0.shape)
    c = rng.standard_normal(x0.shape)
    x1, v1, _ = oracle.be_step(m, x0, v0, p.a, rtol=1e-13)
    ms = m.replace(xhat=x0 + m.h * v0, x0=x0)
    lam, _ = ms.adjoint(x1, p.a, c)
    vjps = ms.material_vjp(x1, lam, p.a)
    for name, v in zip(("mu", "lam", "k_muscle"), vjps):
        th = getattr(m, name)
        eps = 1e-5 * th
        xp, _, _ = oracle.be_step(m.replace(**{name: th + eps}), x0, v0, p.a, rtol=1e-13)
        xm, _, _ = oracle.be_step(m.replace(**{name: th - eps}), x0, v0, p.a, rtol=1e-13)
        fd = np.sum(c * (xp - xm)) / (2 * eps)
        assert math.isclose(fd, v.sum(), rel_tol=1e-5), name


def test_rollout_material_gradient_matches_fd():
    """BPTT material gradient of a 3-step rollout (sum over steps of the
    per-step material VJPs) vs central FD of the rollout's loss."""
    p = synth.make_small2d(4, 2, fix_bottom=False)
    p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
    p.k_friction = 2e3
    m = oracle.make_model(p)
    rng = np.random.default_rng(63)
    a_seq = rng.uniform(0.0, 1.0, size=(3, p.n_elem))
    x0 = p.X.copy()
    v0 = 0.2 * rng.standard_normal(x0.shape)
    c = rng.standard_normal(x0.shape)
    xs, vs = oracle.rollout(m, x0, v0, a_seq, rtol=1e-13)
    _, _, _, mat = oracle.rollout_backward(m, xs, vs, a_seq, c, np.zeros_like(c), material=True)
    for name, v in zip(("mu", "lam", "k_muscle"), mat):
        th = getattr(m, name)
        eps = 1e-5 * th
        xp, _ = oracle.rollout(m.replace(**{name: th + eps}), x0, v0, a_seq, rtol=1e-13)
        xm, _ = oracle.rollout(m.replace(**{name: th - eps}), x0, v0, a_seq, rtol=1e-13)
        fd = np.sum(c * (xp[-1] - xm[-1])) / (2 * eps)
        assert math.isclose(fd, v, rel_tol=1e-5), name
