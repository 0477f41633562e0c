"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (stated once, used below):

* FP64 kernels: energy within 1e-12 of the sum of |terms|; forces within
  1e-12 of the largest per-entry sum of |element contributions| (plain
  per-vertex relative error is meaningless where element forces cancel);
  HVP and VJP within 1e-12 of their largest entry.
* FP32 kernels (mixed precision): HVP within 1e-5 of its largest entry,
  computed with the same FP32-rounded direction on both sides.
* Converged states: the oracle's own gradient at the GPU state meets the
  Newton tolerance |g| <= 1e-8 |g0| (up to 1% slack for the different sum
  order), and the states agree to 1e-5 of the displacement.
* dL/da: relative L2 error <= 1e-4 (mixed) or <= 1e-7 (FP64 path).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from simhelp import deformed, dev, host, make_sim

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def _problems():
    return {
        "c1": synth.make_config1,
        "small3d_t5": lambda: synth.make_small3d(6, 4, 4, split=5, seed=21),
        "small3d_t6": lambda: synth.make_small3d(6, 4, 4, split=6, seed=22),
    }


@pytest.fixture(params=sorted(_problems()))
def prob(request):
    return _problems()[request.param]()


# --------------------------------------------------------------- element kernels

@pytest.mark.parametrize("tile_elems", [0, 24])
@pytest.mark.parametrize("log_mode", [0, 1])
def test_energy_and_gradient_fp64(prob, tile_elems, log_mode):
    prob.log_mode = log_mode
    sim = make_sim(prob, "fp64", tile_elems=tile_elems)
    m = oracle.make_model(prob)
    x = deformed(prob, 0.03, seed=1)
    E, g = sim.energy_grad(dev(x), dev(prob.a))
    E_or, S_or = m.energy(x, prob.a, with_abs=True)
    g_or, scale = m.grad(x, prob.a, with_scale=True)
    assert abs(float(E) - E_or) <= TOL64 * S_or
    assert np.abs(host(g) - g_or).max() <= TOL64 * scale.max()
    if tile_elems:
        assert sim.tile_stats()["n_tiles"] > 4  # the halo path is exercised


def test_gradient_mixed_handle_is_fp64(prob):
    sim = make_sim(prob, "mixed")
    m = oracle.make_model(prob)
    x = deformed(prob, 0.03, seed=2)
    E, g = sim.energy_grad(dev(x), dev(prob.a))
    g_or, scale = m.grad(x, prob.a, with_scale=True)
    assert np.abs(host(g) - g_or).max() <= TOL64 * scale.max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("tile_elems", [0, 24])
def test_hvp(prob, precision, tile_elems):
    sim = make_sim(prob, precision, tile_elems=tile_elems, k_contact=1e5)
    prob.k_contact = 1e5
    m = oracle.make_model(prob)
    x = deformed(prob, 0.03, seed=3)
    x[:, 1] -= 0.01  # some vertices below the ground: the contact stiffness is active
    x[prob.fixed.astype(bool)] = prob.X[prob.fixed.astype(bool)]
    rng = np.random.default_rng(4)
    v = rng.standard_normal(x.shape)
    if precision == "mixed":
        v = v.astype(np.float32).astype(np.float64)
    Hv = host(sim.hvp(dev(x), dev(prob.a), dev(v, sim.vec_dtype))).astype(np.float64)
    Hv_or = m.hvp(x, prob.a, v)
    tol = TOL64 if precision == "fp64" else TOL32
    assert np.abs(Hv - Hv_or).max() <= tol * np.abs(Hv_or).max()


def test_hvp_is_deterministic(prob):
    sim = make_sim(prob, "mixed", tile_elems=24)
    x = dev(deformed(prob, 0.03, seed=5))
    v = dev(np.random.default_rng(6).standard_normal(prob.X.shape), torch.float32)
    a = dev(prob.a)
    h1 = sim.hvp(x, a, v)
    h2 = sim.hvp(x, a, v)
    assert torch.equal(h1, h2)


def test_param_vjp_fp64(prob):
    sim = make_sim(prob, "fp64")
    m = oracle.make_model(prob)
    x = deformed(prob, 0.03, seed=7)
    lam = np.random.default_rng(8).standard_normal(x.shape)
    lam[prob.fixed.astype(bool)] = 0.0
    out = host(sim.param_vjp(dev(x), dev(prob.a), dev(lam)))
    ref = m.param_vjp(x, lam)
    assert np.abs(out - ref).max() <= TOL64 * np.abs(ref).max()


# --------------------------------------------------------------- solves

def _solve_and_check(p, precision, **kw):
    sim = make_sim(p, precision, **kw)
    m = oracle.make_model(p)
    a = dev(p.a)
    x, st = sim.solve(a)
    assert st["status"] == 0, st
    xg = host(x)
    g0 = np.linalg.norm(m.grad(p.X, p.a))
    g_at = np.linalg.norm(m.grad(xg, p.a))
    assert g_at <= 1.01e-8 * g0 + 1e-13 * g0, (g_at / g0, st)
    return sim, m, x, xg, st


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_quasistatic_solve_and_gradient_c1(precision):
    p = synth.make_config1()
    sim, m, x, xg, st = _solve_and_check(p, precision, adjoint_rtol=1e-10 if precision == "fp64" else 1e-6)
    x_or, st_or = m.newton(p.a, rtol=1e-8)
    disp = np.abs(x_or - p.X).max()
    assert np.abs(xg - x_or).max() <= 1e-5 * disp
    # adjoint + parameter VJP
    gL = oracle.mean_loss_grad(xg, p.target)
    lam, st_a = sim.adjoint(x, dev(p.a), dev(gL))
    dLda = host(sim.param_vjp(x, dev(p.a), lam))
    _, _, dLda_or, _ = oracle.quasistatic_forward_backward(m, p.a, p.target, rtol=1e-10)
    err = np.linalg.norm(dLda - dLda_or) / np.linalg.norm(dLda_or)
    assert err <= (1e-7 if precision == "fp64" else 1e-4), err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_quasistatic_solve_and_gradient_3d(precision):
    p = synth.make_small3d(8, 4, 4, split=5, seed=31)
    sim, m, x, xg, st = _solve_and_check(p, precision, tile_elems=128,
                                         adjoint_rtol=1e-10 if precision == "fp64" else 1e-6)
    gL = oracle.mean_loss_grad(xg, p.target)
    lam, _ = sim.adjoint(x, dev(p.a), dev(gL))
    dLda = host(sim.param_vjp(x, dev(p.a), lam))
    _, _, dLda_or, _ = oracle.quasistatic_forward_backward(m, p.a, p.target, rtol=1e-10)
    err = np.linalg.norm(dLda - dLda_or) / np.linalg.norm(dLda_or)
    assert err <= (1e-7 if precision == "fp64" else 1e-4), err


def test_config3_full_size_properties():
    """Config 3 (40,960 tets): forward residual and adjoint residual checked by
    the oracle at the GPU's solution; dL/da checked against the oracle's VJP at
    the GPU's (x*, lambda)."""
    p = synth.make_config3()
    sim, m, x, xg, st = _solve_and_check(p, "mixed")
    gL = oracle.mean_loss_grad(xg, p.target)
    lam, st_a = sim.adjoint(x, dev(p.a), dev(gL))
    assert st_a["status"] == 0, st_a
    lg = host(lam)
    b = gL.copy()
    b[p.fixed.astype(bool)] = 0.0
    res = np.linalg.norm(m.hvp(xg, p.a, lg) - b) / np.linalg.norm(b)
    assert res <= 1e-4, res
    dLda = host(sim.param_vjp(x, dev(p.a), lam))
    ref = m.param_vjp(xg, lg)
    assert np.abs(dLda - ref).max() <= TOL64 * np.abs(ref).max()


def test_autograd_quasistatic_layer():
    from paper_2102_05791_gb300.api import QuasistaticSolve
    p = synth.make_config1()
    sim = make_sim(p, "fp64", adjoint_rtol=1e-10)
    a = dev(p.a).requires_grad_(True)
    x = QuasistaticSolve.apply(sim, a)
    tgt = dev(p.target)
    L = 0.5 * ((x.mean(dim=0) - tgt) ** 2).sum()
    L.backward()
    m = oracle.make_model(p)
    _, _, dLda_or, _ = oracle.quasistatic_forward_backward(m, p.a, p.target, rtol=1e-10)
    err = np.linalg.norm(host(a.grad) - dLda_or) / np.linalg.norm(dLda_or)
    assert err <= 1e-7, err


# --------------------------------------------------------------- dynamics

def _dyn(nx=8, ny=4):
    p = synth.make_small2d(nx, ny, fix_bottom=False, seed=41)
    p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
    return p


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_be_step_and_backward(precision):
    p = _dyn()
    sim = make_sim(p, precision, tile_elems=16, adjoint_rtol=1e-10 if precision == "fp64" else 1e-7)
    m = oracle.make_model(p)
    rng = np.random.default_rng(42)
    x0 = p.X.copy()
    v0 = 0.3 * rng.standard_normal(x0.shape)
    x1, v1, st = sim.step(dev(x0), dev(v0), dev(p.a))
    assert st["status"] == 0
    x1_or, v1_or, _ = oracle.be_step(m, x0, v0, p.a, rtol=1e-10)
    scale = np.abs(x1_or - x0).max()
    assert np.abs(host(x1) - x1_or).max() <= 1e-5 * scale
    xb1 = rng.standard_normal(x0.shape)
    vb1 = rng.standard_normal(x0.shape)
    xb0, vb0, ab, _ = sim.step_backward(dev(x0), dev(v0), x1, dev(p.a), dev(xb1), dev(vb1))
    xb0_or, vb0_or, ab_or = oracle.be_step_backward(m, x0, v0, host(x1), p.a, xb1, vb1)
    tol = 1e-7 if precision == "fp64" else 1e-4
    for got, ref in ((xb0, xb0_or), (vb0, vb0_or), (ab, ab_or)):
        assert np.linalg.norm(host(got) - ref) <= tol * np.linalg.norm(ref)


def test_rollout_bptt_matches_oracle_and_checkpointing_is_exact():
    p = _dyn(6, 3)
    sim = make_sim(p, "fp64", tile_elems=12, adjoint_rtol=1e-11)
    m = oracle.make_model(p)
    rng = np.random.default_rng(43)
    nT = 5
    a_seq = rng.uniform(0.0, 1.0, size=(nT, p.n_elem))
    x0, v0 = p.X.copy(), np.zeros_like(p.X)
    xT, vT, ck, st = sim.rollout(dev(x0), dev(v0), dev(a_seq), ckpt_every=2)
    xs, vs = oracle.rollout(m, x0, v0, a_seq, rtol=1e-8)
    assert np.abs(host(xT) - xs[-1]).max() <= 1e-6 * np.abs(xs[-1] - x0).max()
    c = rng.standard_normal(x0.shape)
    xb0, vb0, ab, _ = sim.rollout_backward(dev(a_seq), ck, 2, dev(c), dev(np.zeros_like(c)))
    xb0_or, vb0_or, ab_or = oracle.rollout_backward(m, xs, vs, a_seq, c, np.zeros_like(c))
    assert np.linalg.norm(host(ab) - ab_or) <= 1e-6 * np.linalg.norm(ab_or)
    assert np.linalg.norm(host(vb0) - vb0_or) <= 1e-6 * np.linalg.norm(vb0_or)
    # recomputation from checkpoints is deterministic: ckpt_every 1 and 2 agree bit for bit
    xT1, vT1, ck1, _ = sim.rollout(dev(x0), dev(v0), dev(a_seq), ckpt_every=1)
    assert torch.equal(xT1, xT)
    xb0_1, vb0_1, ab_1, _ = sim.rollout_backward(dev(a_seq), ck1, 1, dev(c), dev(np.zeros_like(c)))
    assert torch.equal(ab_1, ab) and torch.equal(xb0_1, xb0)


# --------------------------------------------------------------- errors and edge cases

def test_single_element_meshes():
    for d in (2, 3):
        X = np.vstack([np.zeros(d), np.eye(d)])
        T = np.arange(d + 1, dtype=np.int32)[None, :]
        fib = np.zeros((1, d))
        fib[0, 0] = 1.0
        p = synth.SynthProblem("one", d, X, T, np.zeros(d + 1, np.uint8), fib, np.array([0.5]), np.zeros(d))
        sim = make_sim(p, "fp64")
        m = oracle.make_model(p)
        x = X + 0.1 * np.random.default_rng(d).standard_normal(X.shape)
        E, g = sim.energy_grad(dev(x), dev(p.a))
        g_or, sc = m.grad(x, p.a, with_scale=True)
        assert np.abs(host(g) - g_or).max() <= TOL64 * sc.max()


def test_rejects_bad_meshes():
    from paper_2102_05791_gb300.api import SimError
    p = synth.make_small2d(2, 1)
    T = p.T.copy()
    T[0, [1, 2]] = T[0, [2, 1]]  # flip one triangle
    with pytest.raises(SimError) as e:
        make_sim(synth.SynthProblem("bad", 2, p.X, T, p.fixed, p.fiber, p.a, p.target), "fp64")
    assert e.value.code == -3
    T = p.T.copy()
    T[0, 0] = p.n_vert
    with pytest.raises(SimError) as e:
        make_sim(synth.SynthProblem("bad", 2, p.X, T, p.fixed, p.fiber, p.a, p.target), "fp64")
    assert e.value.code == -1


def test_inverted_state_gives_infinite_energy():
    p = synth.make_small2d(2, 1)
    sim = make_sim(p, "fp64")
    x = p.X.copy()
    x[:, 0] *= -1.0  # mirror: every triangle inverted
    E, _ = sim.energy_grad(dev(x), dev(p.a))
    assert math.isinf(float(E))


def test_iteration_cap_reports_not_converged():
    p = synth.make_config1()
    sim = make_sim(p, "fp64", max_newton=1)
    x, st = sim.solve(dev(p.a), check=False)
    assert st["status"] == -4 and st["newton_iters"] == 1


def test_mixed_cg_iterations_track_fp64():
    """The FP32 CG loop (FP32 step lengths and compensated FP32 sums) takes
    about as many iterations as the FP64 one on the same solves; a broken
    step length or direction update shows up here as a large excess."""
    p = synth.make_small3d(8, 4, 4, split=5, seed=31)
    its = {}
    for precision in ("fp64", "mixed"):
        sim = make_sim(p, precision, tile_elems=128, adjoint_rtol=1e-6)
        a = dev(p.a)
        x, st = sim.solve(a)
        assert st["status"] == 0, st
        gL = oracle.mean_loss_grad(host(x), p.target)
        _, sta = sim.adjoint(x, a, dev(gL))
        its[precision] = (st["cg_iters_total"], sta["cg_iters_total"])
        sim.close()
    for k in range(2):
        assert its["mixed"][k] <= 1.25 * its["fp64"][k] + 10, its
