"""The paper's active-spring muscle (Eq. active-spring-potential,
(k/2)(|F f|/a - 1)^2 per element) on the GPU vs the oracle: energy,
gradient, HVP, parameter VJP, quasistatic solves with their gradients, a
backward-Euler step with its backward, and the batched solver.

Tolerances as in the contractile parity tests: FP64 kernels within 1e-12 of
the sum of |terms| (energy), of the per-entry |contribution| scale
(gradient) or of the largest entry (HVP, VJP); FP32 HVP within 1e-5 of its
largest entry; converged states within 1e-5 of the displacement; dL/da
relative L2 within 1e-7 (FP64) or 1e-4 (mixed)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from simhelp import deformed, dev, host, make_sim

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def _spring(p):
    p.muscle_model = 1
    p.a = 0.5 + 0.5 * p.a  # actions in [0.5, 1]: contraction to half length at most
    return p


def _problems():
    return {
        "c1": lambda: _spring(synth.make_config1()),
        "small3d_t5": lambda: _spring(synth.make_small3d(6, 4, 4, split=5, seed=21)),
    }


@pytest.fixture(params=sorted(_problems()))
def prob(request):
    return _problems()[request.param]()


def _sim(p, precision, **kw):
    return make_sim(p, precision, muscle_model=1, **kw)


@pytest.mark.parametrize("tile_elems", [0, 24])
def test_spring_energy_and_gradient_fp64(prob, tile_elems):
    sim = _sim(prob, "fp64", tile_elems=tile_elems)
    m = oracle.make_model(prob)
    assert m.muscle_model == 1
    x = deformed(prob, 0.03, seed=1)
    E, g = sim.energy_grad(dev(x), dev(prob.a))
    E_or, S_or = m.energy(x, prob.a, with_abs=True)
    g_or, scale = m.grad(x, prob.a, with_scale=True)
    assert abs(float(E) - E_or) <= TOL64 * S_or
    assert np.abs(host(g) - g_or).max() <= TOL64 * scale.max()
    # the model differs from the contractile one by far more than the tolerance
    g_c = m.replace(muscle_model=0).grad(x, prob.a)
    assert np.abs(g_c - g_or).max() > 1e-3 * np.abs(g_or).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("tile_elems", [0, 24])
def test_spring_hvp(prob, precision, tile_elems):
    sim = _sim(prob, precision, tile_elems=tile_elems)
    m = oracle.make_model(prob)
    x = deformed(prob, 0.03, seed=3)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(x.shape)
    if precision == "mixed":
        v = v.astype(np.float32).astype(np.float64)
    Hv = host(sim.hvp(dev(x), dev(prob.a), dev(v, sim.vec_dtype))).astype(np.float64)
    Hv_or = m.hvp(x, prob.a, v)
    tol = TOL64 if precision == "fp64" else TOL32
    assert np.abs(Hv - Hv_or).max() <= tol * np.abs(Hv_or).max()


def test_spring_param_vjp_fp64(prob):
    sim = _sim(prob, "fp64", tile_elems=24)
    m = oracle.make_model(prob)
    x = deformed(prob, 0.03, seed=7)
    lam = np.random.default_rng(8).standard_normal(x.shape)
    lam[prob.fixed.astype(bool)] = 0.0
    out = host(sim.param_vjp(dev(x), dev(prob.a), dev(lam)))
    ref = m.param_vjp(x, lam, prob.a)
    assert np.abs(out - ref).max() <= TOL64 * np.abs(ref).max()


@pytest.mark.parametrize("kind", ["c1", "3d"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spring_quasistatic_solve_and_gradient(kind, precision):
    p = _spring(synth.make_config1() if kind == "c1" else synth.make_small3d(8, 4, 4, split=5, seed=31))
    sim = _sim(p, precision, tile_elems=0 if kind == "c1" else 128,
               adjoint_rtol=1e-10 if precision == "fp64" else 1e-6)
    m = oracle.make_model(p)
    a = dev(p.a)
    x, st = sim.solve(a)
    assert st["status"] == 0, st
    xg = host(x)
    g0 = np.linalg.norm(m.grad(p.X, p.a))
    assert np.linalg.norm(m.grad(xg, p.a)) <= 1.01e-8 * g0 + 1e-13 * g0
    x_or, _ = m.newton(p.a, rtol=1e-8)
    assert np.abs(xg - x_or).max() <= 1e-5 * np.abs(x_or - p.X).max()
    gL = oracle.mean_loss_grad(xg, p.target)
    lam, _ = sim.adjoint(x, a, dev(gL))
    dLda = host(sim.param_vjp(x, a, lam))
    _, _, dLda_or, _ = oracle.quasistatic_forward_backward(m, p.a, p.target, rtol=1e-10)
    err = np.linalg.norm(dLda - dLda_or) / np.linalg.norm(dLda_or)
    assert err <= (1e-7 if precision == "fp64" else 1e-4), err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spring_be_step_and_backward(precision):
    p = _spring(synth.make_small2d(8, 4, fix_bottom=False, seed=41))
    p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
    sim = _sim(p, precision, tile_elems=16, adjoint_rtol=1e-10 if precision == "fp64" else 1e-7)
    m = oracle.make_model(p)
    rng = np.random.default_rng(42)
    x0 = p.X.copy()
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


def test_spring_batch_matches_oracle():
    from paper_2102_05791_gb300.api import Batch
    probs = []
    for i, (nx, ny, mu) in enumerate([(4, 2, 1e4), (7, 3, 7e3), (5, 2, 1.6e4)]):
        p = synth.make_small2d(nx, ny, fix_bottom=False, seed=80 + i)
        p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
        p.mu, p.lam = mu, 4.0 * mu
        p.muscle_model = 1
        probs.append(p)
    b = Batch(probs, adjoint_rtol=1e-8)
    rng = np.random.default_rng(83)
    nT = 3
    a_seq = rng.uniform(0.5, 1.0, size=(nT, b.E))
    x0 = np.concatenate([p.X for p in probs])
    v0 = 0.1 * rng.standard_normal(x0.shape)
    xbT = rng.standard_normal(x0.shape)
    vbT = 0.01 * rng.standard_normal(x0.shape)
    sx, sv, abar, xb0, vb0, ms = b.rollout(dev(x0), dev(v0), dev(a_seq), dev(xbT), dev(vbT))
    torch.cuda.synchronize()
    ms = host(ms)
    assert (ms[:, 0] == 0).all(), ms
    sx, abar, xb0, vb0 = host(sx), host(abar), host(xb0), host(vb0)
    vo, eo = b.vert_offsets, b.elem_offsets
    for i, p in enumerate(probs):
        m = oracle.make_model(p)
        vs_, ve_ = vo[i], vo[i + 1]
        es_, ee_ = eo[i], eo[i + 1]
        a_i = a_seq[:, es_:ee_]
        xs, vs = oracle.rollout(m, x0[vs_:ve_], v0[vs_:ve_], a_i, rtol=1e-10)
        assert np.abs(sx[-1, vs_:ve_] - xs[-1]).max() <= 1e-6 * np.abs(xs[-1] - xs[0]).max()
        xb, vb, ab = oracle.rollout_backward(m, xs, vs, a_i, xbT[vs_:ve_], vbT[vs_:ve_])
        assert np.linalg.norm(abar[:, es_:ee_] - ab) <= 1e-4 * np.linalg.norm(ab)
        assert np.linalg.norm(vb0[vs_:ve_] - vb) <= 1e-4 * np.linalg.norm(vb)
        assert np.linalg.norm(xb0[vs_:ve_] - xb) <= 1e-4 * np.linalg.norm(xb)
    b.close()


def test_spring_rejects_mixed_muscle_models_in_a_batch():
    from paper_2102_05791_gb300.api import Batch, SimError
    probs = []
    for i in range(2):
        p = synth.make_small2d(4, 2, fix_bottom=False, seed=90 + i)
        p.dt = 1.0 / 30.0
        p.muscle_model = i
        probs.append(p)
    with pytest.raises(SimError):
        Batch(probs)
