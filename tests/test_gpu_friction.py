"""Ground friction (Sec. 4.2) on the GPU vs the oracle: one backward-Euler
step and its backward, a checkpointed rollout with BPTT, the batched
persistent solver, and a full-size 64 x 32 walker rollout.

Tolerances as for the frictionless dynamics: states within 1e-5 (single
step) or 1e-6 (rollouts) of the displacement scale; gradients within 1e-7
relative L2 in FP64 and 1e-4 in mixed precision (FP64-refined adjoints)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from simhelp import dev, host, make_sim

pytestmark = pytest.mark.gpu

K_F, EPS_F = 2e3, 0.01


def _fric(kind="tri", seed=51, cpow=3):
    if kind == "tri":
        p = synth.make_small2d(8, 4, fix_bottom=False, seed=seed)
    else:
        p = synth.make_small3d(3, 2, 3, split=6, fix_bottom=False, seed=seed)
    # cpow 2 is the paper's one-sided quadratic collision k_c ReLU(-y)^2
    p.k_contact, p.contact_power, p.dt = (1e6 if cpow == 3 else 1e5), cpow, 1.0 / 30.0
    p.k_friction, p.eps_friction = K_F, EPS_F
    return p


def _sim(p, precision, **kw):
    return make_sim(p, precision, k_friction=p.k_friction, eps_friction=p.eps_friction, **kw)


def _start(p, rng):
    x0 = p.X + 0.002 * rng.standard_normal(p.X.shape)
    x0[:, 1] += 0.004
    v0 = 0.3 * rng.standard_normal(x0.shape)
    return x0, v0


@pytest.mark.parametrize("cpow", [2, 3])
@pytest.mark.parametrize("kind", ["tri", "tet"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_friction_step_and_backward(kind, precision, cpow):
    p = _fric(kind, cpow=cpow)
    sim = _sim(p, precision, tile_elems=16, adjoint_rtol=1e-10 if precision == "fp64" else 1e-7)
    m = oracle.make_model(p)
    rng = np.random.default_rng(52)
    x0, v0 = _start(p, rng)
    assert (x0[:, 1] < EPS_F).any() and (x0[:, 1] > EPS_F).any()
    x1, v1, st = sim.step(dev(x0), dev(v0), dev(p.a))
    assert st["status"] == 0, st
    x1_or, v1_or, _ = oracle.be_step(m, x0, v0, p.a, rtol=1e-10)
    scale = np.abs(x1_or - x0).max()
    assert np.abs(host(x1) - x1_or).max() <= 1e-5 * scale
    # friction changed the answer well beyond the tolerance
    x1_nf, _, _ = oracle.be_step(m.replace(k_friction=0.0), x0, v0, p.a, rtol=1e-10)
    assert np.abs(x1_nf - x1_or).max() > 1e-2 * scale
    xb1 = rng.standard_normal(x0.shape)
    vb1 = rng.standard_normal(x0.shape)
    xb0, vb0, ab, _ = sim.step_backward(dev(x0), dev(v0), x1, dev(p.a), dev(xb1), dev(vb1))
    xb0_or, vb0_or, ab_or = oracle.be_step_backward(m, x0, v0, host(x1), p.a, xb1, vb1)
    tol = 1e-7 if precision == "fp64" else 1e-4
    for got, ref in ((xb0, xb0_or), (vb0, vb0_or), (ab, ab_or)):
        assert np.linalg.norm(host(got) - ref) <= tol * np.linalg.norm(ref)


def test_friction_weights_zero_is_bitwise_frictionless():
    """All vertices start above eps: the friction handle reproduces the
    frictionless one bit for bit (zero weights add exact zeros)."""
    p = _fric()
    rng = np.random.default_rng(53)
    x0, v0 = _start(p, rng)
    x0[:, 1] += 1.0
    a = dev(p.a)
    s1 = _sim(p, "mixed", tile_elems=16)
    s0 = make_sim(p, "mixed", tile_elems=16)
    x1a, v1a, _ = s1.step(dev(x0), dev(v0), a)
    x1b, v1b, _ = s0.step(dev(x0), dev(v0), a)
    assert torch.equal(x1a, x1b) and torch.equal(v1a, v1b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_friction_rollout_bptt(precision):
    p = _fric(seed=54)
    sim = _sim(p, precision, tile_elems=12, adjoint_rtol=1e-11 if precision == "fp64" else 1e-8)
    m = oracle.make_model(p)
    rng = np.random.default_rng(55)
    nT = 5
    a_seq = rng.uniform(0.0, 1.0, size=(nT, p.n_elem))
    x0, v0 = _start(p, rng)
    xT, vT, ck, st = sim.rollout(dev(x0), dev(v0), dev(a_seq), ckpt_every=2)
    assert st["status"] == 0, st
    xs, vs = oracle.rollout(m, x0, v0, a_seq, rtol=1e-10)
    assert np.abs(host(xT) - xs[-1]).max() <= 1e-6 * np.abs(xs[-1] - x0).max()
    c = rng.standard_normal(x0.shape)
    cv = 0.01 * rng.standard_normal(x0.shape)
    xb0, vb0, ab, _ = sim.rollout_backward(dev(a_seq), ck, 2, dev(c), dev(cv))
    xb0_or, vb0_or, ab_or = oracle.rollout_backward(m, xs, vs, a_seq, c, cv)
    tol = 1e-6 if precision == "fp64" else 1e-4
    for got, ref in ((xb0, xb0_or), (vb0, vb0_or), (ab, ab_or)):
        assert np.linalg.norm(host(got) - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("cpow", [2, 3])
def test_friction_batch_matches_oracle(cpow):
    from paper_2102_05791_gb300.api import Batch
    probs = []
    for i, (nx, ny, mu) in enumerate([(4, 2, 1e4), (7, 3, 7e3), (5, 2, 1.6e4)]):
        p = synth.make_small2d(nx, ny, fix_bottom=False, seed=56 + i)
        p.k_contact, p.contact_power, p.dt = (1e6 if cpow == 3 else 1e5), cpow, 1.0 / 30.0
        p.k_friction, p.eps_friction = K_F, EPS_F
        p.mu, p.lam = mu, 4.0 * mu
        probs.append(p)
    b = Batch(probs, adjoint_rtol=1e-8)
    rng = np.random.default_rng(59)
    nT = 3
    a_seq = rng.uniform(0.0, 1.0, size=(nT, b.E))
    starts = [_start(p, rng) for p in probs]
    x0 = np.concatenate([s[0] for s in starts])
    v0 = np.concatenate([s[1] for s in starts])
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
        assert m.k_friction == K_F
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


def test_friction_config2_walker_rollout():
    """64 x 32 walker (4,096 triangles) with friction on: 12 steps of the
    group-activation gait, state and per-group gradient vs the oracle."""
    nT = 12
    p = synth.make_config2(n_steps=nT)
    p.k_friction, p.eps_friction = K_F, EPS_F
    group = p.extra["group"]
    a_seq = p.extra["a_groups"][:, group]
    sim = _sim(p, "mixed", adjoint_rtol=1e-8)
    x0, v0 = p.X.copy(), np.zeros_like(p.X)
    xT, vT, ck, st = sim.rollout(dev(x0), dev(v0), dev(a_seq), ckpt_every=4)
    assert st["status"] == 0, st
    m = oracle.make_model(p)
    xs, vs = oracle.rollout(m, x0, v0, a_seq, rtol=1e-10)
    assert np.abs(host(xT) - xs[-1]).max() <= 1e-6 * np.abs(xs[-1] - xs[0]).max()
    xbT = np.zeros_like(x0)
    xbT[:, 0] = 1.0 / p.n_vert
    xb0, vb0, ab, _ = sim.rollout_backward(dev(a_seq), ck, 4, dev(xbT), dev(np.zeros_like(x0)))
    _, _, ab_or = oracle.rollout_backward(m, xs, vs, a_seq, xbT, np.zeros_like(x0))
    g_gpu = np.stack([np.bincount(group, weights=host(ab)[t], minlength=8) for t in range(nT)])
    g_or = np.stack([np.bincount(group, weights=ab_or[t], minlength=8) for t in range(nT)])
    assert np.linalg.norm(g_gpu - g_or) <= 1e-4 * np.linalg.norm(g_or)
    # with friction the walker's horizontal mean moves: its gradient is not degenerate
    assert np.abs(g_or).max() > 0.0
