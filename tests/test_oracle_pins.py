"""Pins for the FP64 oracle: checks against facts fixed by the paper and by
mathematics, not against the oracle's own formulas.

Each test names the property it pins and the passage that fixes it.  A wrong
sign, a dropped term or a transposed operand anywhere in the oracle's energy,
gradient, HVP, VJP, Newton or adjoint makes at least one of these fail.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _no_gravity(m):
    return m.replace(gravity=0.0, k_contact=0.0)


def _rand_x(p, rng, amp=0.05):
    return p.X + amp * rng.standard_normal(p.X.shape)


def _rotation(d, rng):
    A = rng.standard_normal((d, d))
    Q, R = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


PROBS = {
    "tri": lambda: synth.make_small2d(4, 2),
    "tet5": lambda: synth.make_small3d(2, 2, 2, split=5),
    "tet6": lambda: synth.make_small3d(2, 2, 2, split=6, seed=13),
}


@pytest.fixture(params=sorted(PROBS))
def prob(request):
    return PROBS[request.param]()


@pytest.fixture(params=[0, 1], ids=["exactlog", "quadlog"])
def log_mode(request):
    return request.param


# --------------------------------------------------------------- rest state

def test_rest_energy_and_gradient_vanish(prob, log_mode):
    """Psi(I) = 0 and P(I) = 0 (Eq. neohookean-psi at F = I), muscle off, no gravity."""
    m = _no_gravity(oracle.make_model(prob, log_mode=log_mode, with_fixed=False))
    a0 = np.zeros(prob.n_elem)
    assert abs(m.energy(prob.X, a0)) < 1e-9
    assert np.abs(m.grad(prob.X, a0)).max() < 1e-8
    # an active muscle is not at rest in the reference shape
    assert m.energy(prob.X, np.ones(prob.n_elem)) > 0.0


def test_mesh_measures_closed_form():
    """Sum of W_e is the area / volume of the domain; lumped masses sum to rho * volume."""
    p2 = synth.make_small2d(4, 2)
    m2 = oracle.make_model(p2)
    assert math.isclose(m2.W.sum(), 2.0, rel_tol=1e-12)
    assert math.isclose(m2.mass.sum(), 2.0 * p2.density, rel_tol=1e-12)
    p3 = synth.make_small3d(2, 2, 2, split=6)
    m3 = oracle.make_model(p3)
    assert math.isclose(m3.W.sum(), 1.0, rel_tol=1e-12)
    assert math.isclose(m3.mass.sum(), 1.0 * p3.density, rel_tol=1e-12)


# --------------------------------------------------------------- invariances

def test_rotation_and_translation_invariance(prob, log_mode):
    """Elastic + muscle energy depends on x only through F^T F and |F f| (frame indifference)."""
    rng = np.random.default_rng(1)
    m = _no_gravity(oracle.make_model(prob, log_mode=log_mode, with_fixed=False))
    x = _rand_x(prob, rng)
    R = _rotation(prob.dim, rng)
    t = rng.standard_normal(prob.dim)
    E0 = m.energy(x, prob.a)
    E1 = m.energy(x @ R.T + t, prob.a)
    assert abs(E1 - E0) <= 1e-10 * abs(E0)


def test_force_and_torque_balance(prob, log_mode):
    """Translation invariance gives sum_i f_i = 0; rotation invariance gives sum_i x_i x f_i = 0."""
    rng = np.random.default_rng(2)
    m = _no_gravity(oracle.make_model(prob, log_mode=log_mode, with_fixed=False))
    x = _rand_x(prob, rng)
    g, scale = m.grad(x, prob.a, with_scale=True)
    s = scale.max()
    assert np.abs(g.sum(axis=0)).max() < 1e-12 * s * prob.n_vert
    if prob.dim == 2:
        torque = np.sum(x[:, 0] * g[:, 1] - x[:, 1] * g[:, 0])
        assert abs(torque) < 1e-11 * s * prob.n_vert
    else:
        torque = np.cross(x, g).sum(axis=0)
        assert np.abs(torque).max() < 1e-11 * s * prob.n_vert


def test_patch_test_affine_deformation(prob, log_mode):
    """Under x = A X + b every element has the same F, so with uniform fibers
    and activation the interior vertex forces cancel exactly (patch test)."""
    rng = np.random.default_rng(3)
    d = prob.dim
    A = np.eye(d) + 0.1 * rng.standard_normal((d, d))
    x = prob.X @ A.T + rng.standard_normal(d)
    fib = np.zeros((prob.n_elem, d))
    fib[:, 0] = 1.0
    p = synth.SynthProblem(prob.name, d, prob.X, prob.T, prob.fixed, fib, prob.a, prob.target)
    m = _no_gravity(oracle.make_model(p, log_mode=log_mode, with_fixed=False))
    g, scale = m.grad(x, np.full(prob.n_elem, 0.7), with_scale=True)
    # interior vertices: not on the bounding box
    lo, hi = prob.X.min(axis=0), prob.X.max(axis=0)
    interior = np.all((prob.X > lo + 1e-9) & (prob.X < hi - 1e-9), axis=1)
    assert interior.any()
    assert np.abs(g[interior]).max() < 1e-11 * scale.max()


# --------------------------------------------------------------- closed forms

@pytest.mark.parametrize("s", [0.6, 1.0, 1.3, 2.0])
def test_single_element_uniaxial_closed_form(s):
    """One unit right triangle / tet stretched by F = diag(s, 1[, 1]):
    Psi = mu/2 (s^2 - 1) - mu log s + lambda/2 log^2 s, and dPsi/ds is the
    force on the stretched vertex (Eq. neohookean-psi, exact log)."""
    mu, lam, k, act = 1.0e4, 4.0e4, 5.0e3, 0.3
    for d in (2, 3):
        X = np.vstack([np.zeros(d), np.eye(d)])
        T = np.arange(d + 1, dtype=np.int32)[None, :]
        fib = np.zeros((1, d))
        fib[0, 0] = 1.0
        p = synth.SynthProblem("unit", d, X, T, np.zeros(d + 1, np.uint8), fib, np.array([act]),
                               np.zeros(d), mu=mu, lam=lam, k_muscle=k, gravity=0.0)
        m = oracle.make_model(p, with_fixed=False)
        x = X.copy()
        x[1, 0] = s
        W = 1.0 / math.factorial(d)
        psi = 0.5 * mu * (s * s - 1.0) - mu * math.log(s) + 0.5 * lam * math.log(s) ** 2
        psim = 0.5 * k * act * s * s
        assert math.isclose(m.energy(x, p.a), W * (psi + psim), rel_tol=1e-13, abs_tol=1e-10)
        dpsi = mu * s - mu / s + lam * math.log(s) / s + k * act * s
        g = m.grad(x, p.a)
        assert math.isclose(g[1, 0], W * dpsi, rel_tol=1e-12, abs_tol=1e-9)
        assert abs(g[1, 1:]).max() < 1e-9


def test_quadratic_log_matches_taylor_polynomial():
    """QUAD mode: Psi uses q(J) = (J-1) - (J-1)^2/2, which stays finite for J <= 0
    (Sec. 2, quadratic approximation of log for inverted elements)."""
    mu, lam = 1.0e4, 4.0e4
    X = np.vstack([np.zeros(2), np.eye(2)])
    T = np.array([[0, 1, 2]], np.int32)
    p = synth.SynthProblem("unit", 2, X, T, np.zeros(3, np.uint8), np.array([[1.0, 0.0]]),
                           np.zeros(1), np.zeros(2), mu=mu, lam=lam, gravity=0.0, log_mode=1)
    m = oracle.make_model(p, with_fixed=False)
    for s in (1.2, 0.5, -0.5):
        x = X.copy()
        x[1, 0] = s
        J = s
        q = (J - 1) - 0.5 * (J - 1) ** 2
        psi = 0.5 * mu * (s * s - 1.0) - mu * q + 0.5 * lam * q * q
        assert math.isclose(m.energy(x, p.a), 0.5 * psi, rel_tol=1e-13)
    # the exact-log model refuses an inverted element
    me = m.replace(log_mode=0)
    x = X.copy()
    x[1, 0] = -0.5
    assert math.isinf(me.energy(x, p.a))


def test_rest_hessian_is_textbook_cst_stiffness(log_mode):
    """At F = I the Hessian equals the constant-strain-triangle stiffness
    A B^T D B of linear elasticity with the same Lame parameters (golden file)."""
    g = json.load(open(os.path.join(GOLDEN, "cst_plane_strain.json")))
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    p = synth.SynthProblem("cst", 2, X, np.array([[0, 1, 2]], np.int32), np.zeros(3, np.uint8),
                           np.array([[1.0, 0.0]]), np.zeros(1), np.zeros(2),
                           mu=g["mu"], lam=g["lambda"], gravity=0.0, log_mode=log_mode)
    m = oracle.make_model(p, with_fixed=False)
    H = m.dense_hessian(X, np.zeros(1))
    K = np.array(g["K_expected"])
    assert np.abs(H - K).max() < 1e-9 * np.abs(K).max()


def _linear_elastic_stiffness(m):
    """Textbook assembly: K = sum_e W_e B_e^T C B_e, Voigt strains, isotropic C."""
    d, n = m.d, m.nv * m.d
    K = np.zeros((n, n))
    lam, mu = m.lam, m.mu
    nvoigt = 3 if d == 2 else 6
    pairs = [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    D = np.zeros((nvoigt, nvoigt))
    D[:d, :d] = lam
    D[np.arange(d), np.arange(d)] += 2 * mu
    D[np.arange(d, nvoigt), np.arange(d, nvoigt)] = mu
    for e in range(m.ne):
        Bi = m.Dminv[e]
        grads = np.vstack([-Bi.sum(axis=0), Bi])  # gradient of each barycentric shape function
        B = np.zeros((nvoigt, (d + 1) * d))
        for a in range(d + 1):
            for r, (i, j) in enumerate(pairs):
                if i == j:
                    B[r, a * d + i] += grads[a, i]
                else:
                    B[r, a * d + i] += grads[a, j]
                    B[r, a * d + j] += grads[a, i]
        Ke = m.W[e] * B.T @ D @ B
        idx = np.concatenate([np.arange(v * d, v * d + d) for v in m.T[e]])
        K[np.ix_(idx, idx)] += Ke
    return K


def test_rest_hessian_is_linear_elasticity(prob, log_mode):
    """Same pin on jittered meshes in 2D and 3D, assembled from B-matrices."""
    m = _no_gravity(oracle.make_model(prob, log_mode=log_mode, with_fixed=False))
    H = m.dense_hessian(prob.X, np.zeros(prob.n_elem))
    K = _linear_elastic_stiffness(m)
    assert np.abs(H - K).max() < 1e-9 * np.abs(K).max()


def test_muscle_energy_is_exact_quadratic(prob):
    """(k/2) a |F f|^2 is quadratic in x, so E(x+v) - E(x) - g.v = 1/2 v^T H v exactly."""
    rng = np.random.default_rng(4)
    m = _no_gravity(oracle.make_model(prob, with_fixed=False)).replace(mu=0.0, lam=0.0)
    x = _rand_x(prob, rng)
    v = 0.1 * rng.standard_normal(x.shape)
    lhs = m.energy(x + v, prob.a) - m.energy(x, prob.a) - np.sum(m.grad(x, prob.a) * v)
    rhs = 0.5 * np.sum(v * m.hvp(x, prob.a, v))
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)


# --------------------------------------------------------------- derivatives

def test_gradient_matches_central_differences(prob, log_mode):
    """f = -grad E (Eq. f-as-grad): directional derivative vs central FD, with O(eps^2) decay."""
    rng = np.random.default_rng(5)
    m = oracle.make_model(prob, log_mode=log_mode, with_fixed=False).replace(k_contact=1e5)
    x = _rand_x(prob, rng)
    x[:, 1] -= 0.02  # a few vertices below the ground: the contact term is active
    u = rng.standard_normal(x.shape)
    gu = np.sum(m.grad(x, prob.a) * u)
    errs = []
    for eps in (2e-4, 1e-4):
        fd = (m.energy(x + eps * u, prob.a) - m.energy(x - eps * u, prob.a)) / (2 * eps)
        errs.append(abs(fd - gu))
    assert errs[1] < 2e-5 * abs(gu)
    # truncation error of a central difference falls like eps^2
    assert errs[1] < errs[0] / 3.0 or errs[1] < 1e-9 * abs(gu)


def test_hvp_matches_gradient_differences(prob, log_mode):
    """(df/dx) v = d/dx <f, v> (Eq. matrix-free-dfdx): HVP vs central FD of the gradient."""
    rng = np.random.default_rng(6)
    m = oracle.make_model(prob, log_mode=log_mode, with_fixed=False).replace(k_contact=1e5)
    x = _rand_x(prob, rng)
    x[:, 1] -= 0.02
    v = rng.standard_normal(x.shape)
    Hv = m.hvp(x, prob.a, v)
    eps = 1e-6
    fd = (m.grad(x + eps * v, prob.a) - m.grad(x - eps * v, prob.a)) / (2 * eps)
    assert np.abs(Hv - fd).max() < 1e-6 * np.abs(Hv).max()


@pytest.mark.parametrize("power", [2, 3])
def test_contact_penalty_derivatives(power):
    """k_c max(0, -y)^p (Eq. energy-collision for p = 2): energy, force and stiffness."""
    p = synth.make_small2d(3, 1, fix_bottom=False)
    p.k_contact, p.contact_power = 1e5, power
    m = oracle.make_model(p, with_fixed=False).replace(gravity=0.0, mu=0.0, lam=0.0, k_muscle=0.0)
    x = p.X.copy()
    x[:, 1] -= 0.05
    pen = np.maximum(0.0, -x[:, 1])
    assert math.isclose(m.energy(x, p.a), 1e5 * np.sum(pen ** power), rel_tol=1e-13)
    g = m.grad(x, p.a)
    assert np.allclose(g[:, 1], -power * 1e5 * pen ** (power - 1), rtol=1e-13, atol=0)
    v = np.zeros_like(x)
    v[:, 1] = 1.0
    Hv = m.hvp(x, p.a, v)
    expect = power * (power - 1) * 1e5 * np.where(pen > 0, pen ** (power - 2), 0.0)
    assert np.allclose(Hv[:, 1], expect, rtol=1e-13, atol=0)


def test_hessian_symmetric_and_matches_fd(prob, log_mode):
    """H = -df/dx is symmetric (Sec. 3): dense H by HVP columns vs central FD of the gradient."""
    rng = np.random.default_rng(7)
    m = oracle.make_model(prob, log_mode=log_mode)
    x = _rand_x(prob, rng, amp=0.03)
    x[prob.fixed.astype(bool)] = prob.X[prob.fixed.astype(bool)]
    H = m.dense_hessian(x, prob.a)
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()
    n = x.size
    Hfd = np.zeros((n, n))
    eps = 1e-6
    for j in range(n):
        e = np.zeros(n)
        e[j] = eps
        Hfd[:, j] = (m.grad(x + e.reshape(x.shape), prob.a) - m.grad(x - e.reshape(x.shape), prob.a)).ravel() / (2 * eps)
    free = m.free_mask()
    Hff = H[np.ix_(free, free)]
    assert np.abs(Hff - Hfd[np.ix_(free, free)]).max() < 1e-6 * np.abs(Hff).max()
    # pinned rows and columns are dropped
    assert np.abs(H[~free]).max() == 0.0 and np.abs(H[:, ~free]).max() == 0.0
    u, v = rng.standard_normal(x.shape), rng.standard_normal(x.shape)
    assert abs(np.sum(u * m.hvp(x, prob.a, v)) - np.sum(v * m.hvp(x, prob.a, u))) < 1e-10 * np.abs(H).max() * n


def test_param_vjp_matches_mixed_second_derivative(prob):
    """-lambda^T d(grad E)/da_e (Eq. dLda-re-ordered) vs FD of the gradient in a_e."""
    rng = np.random.default_rng(8)
    m = oracle.make_model(prob, with_fixed=False)
    x = _rand_x(prob, rng)
    lam = rng.standard_normal(x.shape)
    vjp = m.param_vjp(x, lam)
    eps = 1e-4
    for e in range(0, prob.n_elem, max(1, prob.n_elem // 7)):
        da = np.zeros(prob.n_elem)
        da[e] = eps
        dg = (m.grad(x, prob.a + da) - m.grad(x, prob.a - da)) / (2 * eps)
        assert math.isclose(vjp[e], -np.sum(lam * dg), rel_tol=1e-7, abs_tol=1e-9 * np.abs(vjp).max())


# --------------------------------------------------------------- solvers

def _tiny_problems():
    return [synth.make_small2d(4, 2), synth.make_small3d(2, 2, 2, split=5)]


@pytest.mark.parametrize("pi", [0, 1])
def test_newton_reaches_a_minimum(pi):
    """x* = argmin E (Eq. x1-quasistatic-argmin): |grad| <= tol, H(x*) positive
    definite on free entries (Sec. 3), same point as a dense Newton iteration."""
    p = _tiny_problems()[pi]
    m = oracle.make_model(p)
    x, st = m.newton(p.a, rtol=1e-10)
    assert st["status"] == oracle.OK
    assert st["res_final"] <= 1e-10 * st["res0"]
    free = m.free_mask()
    H = m.dense_hessian(x, p.a)[np.ix_(free, free)]
    np.linalg.cholesky(H)  # raises unless positive definite
    # dense Newton (numpy solve), full steps from the CG solution's neighbourhood
    xd = p.X.copy()
    for _ in range(200):
        g = m.grad(xd, p.a).ravel()[free]
        if np.linalg.norm(g) <= 1e-10 * st["res0"]:
            break
        Hd = m.dense_hessian(xd, p.a)[np.ix_(free, free)]
        step = np.linalg.solve(Hd, -g)
        t = 1.0
        E0 = m.energy(xd, p.a)
        while True:
            xt = xd.copy()
            xt.reshape(-1)[free] += t * step
            if m.energy(xt, p.a) <= E0 + 1e-4 * t * g @ step + 1e-12 * abs(E0):
                break
            t *= 0.5
        xd = xt
    scale = np.abs(x - p.X).max()
    assert np.abs(xd - x).max() < 1e-7 * scale


@pytest.mark.parametrize("pi", [0, 1])
def test_adjoint_gradient_matches_dense_sensitivity(pi):
    """dL/da = -(H^-1 dL/dx)^T d2E/dx da (Eq. dLda-re-ordered) equals
    dL/dx . dx/da with dx/da = -H^-1 df/da formed densely (Eq. dx1da)."""
    p = _tiny_problems()[pi]
    m = oracle.make_model(p)
    x, lam, dLda, st = oracle.quasistatic_forward_backward(m, p.a, p.target, rtol=1e-11)
    free = m.free_mask()
    H = m.dense_hessian(x, p.a)[np.ix_(free, free)]
    # d(grad)/da column by column, from the closed-form gradient at +-eps
    eps = 1e-5
    G = np.zeros((free.sum(), p.n_elem))
    for e in range(p.n_elem):
        da = np.zeros(p.n_elem)
        da[e] = eps
        G[:, e] = ((m.grad(x, p.a + da) - m.grad(x, p.a - da)).ravel()[free]) / (2 * eps)
    dxda = -np.linalg.solve(H, G)
    gL = oracle.mean_loss_grad(x, p.target).ravel()[free]
    dense = gL @ dxda
    assert np.abs(dense - dLda).max() < 1e-6 * np.abs(dLda).max()


@pytest.mark.parametrize("pi", [0, 1])
def test_adjoint_gradient_matches_fd_through_solve(pi):
    """<dL/da, delta> vs central FD of L(x*(a)) through the whole Newton solve."""
    p = _tiny_problems()[pi]
    m = oracle.make_model(p)
    x, lam, dLda, st = oracle.quasistatic_forward_backward(m, p.a, p.target, rtol=1e-12)
    rng = np.random.default_rng(9)
    delta = rng.standard_normal(p.n_elem)
    eps = 1e-5
    xp, _ = m.newton(p.a + eps * delta, rtol=1e-13)
    xm, _ = m.newton(p.a - eps * delta, rtol=1e-13)
    fd = (oracle.mean_loss(xp, p.target) - oracle.mean_loss(xm, p.target)) / (2 * eps)
    assert math.isclose(fd, float(dLda @ delta), rel_tol=1e-5)


# --------------------------------------------------------------- dynamics

def _dyn_problem():
    p = synth.make_small2d(4, 2, fix_bottom=False)
    p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
    return p


def test_be_step_optimality_and_velocity():
    """x1 solves M (x1 - x0 - h v0) + h^2 grad E(x1) = 0 and v1 = (x1 - x0)/h (Eq. opt-be)."""
    p = _dyn_problem()
    m = oracle.make_model(p)
    rng = np.random.default_rng(10)
    x0 = p.X.copy()
    v0 = 0.3 * rng.standard_normal(x0.shape)
    x1, v1, st = oracle.be_step(m, x0, v0, p.a, rtol=1e-12)
    assert st["status"] == oracle.OK
    # residual of the optimality condition, from the quasistatic model's gradient
    mq = m.replace(h=0.0)
    res = m.mass[:, None] * (x1 - x0 - m.h * v0) + m.h ** 2 * mq.grad(x1, p.a)
    scale = np.abs(m.mass[:, None] * m.h * v0).max() + m.h ** 2 * np.abs(mq.grad(x0, p.a)).max()
    assert np.abs(res).max() < 1e-10 * scale
    assert np.allclose(v1, (x1 - x0) / m.h, rtol=0, atol=1e-15 * np.abs(v1).max() / m.h + 1e-14)


def test_be_step_conserves_momentum_without_external_forces():
    """Internal forces sum to zero, so sum_i m_i v_i is preserved by backward Euler."""
    p = _dyn_problem()
    m = oracle.make_model(p).replace(gravity=0.0, k_contact=0.0)
    rng = np.random.default_rng(11)
    x0 = p.X + 0.02 * rng.standard_normal(p.X.shape)
    v0 = rng.standard_normal(p.X.shape)
    x1, v1, st = oracle.be_step(m, x0, v0, p.a, rtol=1e-12)
    P0 = (m.mass[:, None] * v0).sum(axis=0)
    P1 = (m.mass[:, None] * v1).sum(axis=0)
    assert np.abs(P1 - P0).max() < 1e-9 * np.abs(m.mass[:, None] * v0).sum()


def test_bptt_matches_fd_through_rollout():
    """BPTT through 3 backward-Euler steps vs central FD of the rollout's loss."""
    p = _dyn_problem()
    m = oracle.make_model(p)
    rng = np.random.default_rng(12)
    nT = 3
    a_seq = rng.uniform(0.0, 1.0, size=(nT, p.n_elem))
    x0 = p.X.copy()
    v0 = np.zeros_like(x0)
    xs, vs = oracle.rollout(m, x0, v0, a_seq, rtol=1e-13)
    c = rng.standard_normal(x0.shape)
    cv = rng.standard_normal(x0.shape)

    def loss(xT, vT):
        return float(np.sum(c * xT) + 0.01 * np.sum(cv * vT))

    xbar0, vbar0, abar = oracle.rollout_backward(m, xs, vs, a_seq, c, 0.01 * cv)
    delta = rng.standard_normal(a_seq.shape)
    eps = 1e-5
    xp, vp = oracle.rollout(m, x0, v0, a_seq + eps * delta, rtol=1e-13)
    xm, vm = oracle.rollout(m, x0, v0, a_seq - eps * delta, rtol=1e-13)
    fd = (loss(xp[-1], vp[-1]) - loss(xm[-1], vm[-1])) / (2 * eps)
    assert math.isclose(fd, float(np.sum(abar * delta)), rel_tol=1e-5)
    # and through the initial velocity
    dv = rng.standard_normal(v0.shape)
    xp, vp = oracle.rollout(m, x0, v0 + eps * dv, a_seq, rtol=1e-13)
    xm, vm = oracle.rollout(m, x0, v0 - eps * dv, a_seq, rtol=1e-13)
    fd = (loss(xp[-1], vp[-1]) - loss(xm[-1], vm[-1])) / (2 * eps)
    assert math.isclose(fd, float(np.sum(vbar0 * dv)), rel_tol=1e-5)


def test_mass_weighted_horizontal_centroid_has_zero_gradient():
    """Frictionless ground + internal forces: horizontal momentum is conserved,
    so the mass-weighted horizontal centroid of x_T does not depend on a."""
    p = _dyn_problem()
    m = oracle.make_model(p)
    rng = np.random.default_rng(13)
    a_seq = rng.uniform(0.0, 1.0, size=(3, p.n_elem))
    xs, vs = oracle.rollout(m, p.X.copy(), np.zeros_like(p.X), a_seq, rtol=1e-13)
    xbar = np.zeros_like(p.X)
    xbar[:, 0] = m.mass / m.mass.sum()
    _, _, abar = oracle.rollout_backward(m, xs, vs, a_seq, xbar, np.zeros_like(p.X))
    # compare with the plain-mean gradient, which is not degenerate
    xbar2 = np.zeros_like(p.X)
    xbar2[:, 0] = 1.0 / p.n_vert
    _, _, abar2 = oracle.rollout_backward(m, xs, vs, a_seq, xbar2, np.zeros_like(p.X))
    assert np.abs(abar).max() < 1e-6 * np.abs(abar2).max()
