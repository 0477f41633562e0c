"""Material-parameter VJPs on the GPU (sim_material_vjp) vs the oracle:
per-element dL/dmu, dL/dlambda and dL/dk at a given state and adjoint, in
quasistatic and backward-Euler scaling, both log modes and both muscle
models; and the end-to-end material gradient of a quasistatic solve.

Tolerances: per-element values within 1e-12 of the largest entry (FP64
kernel); solve gradients within 1e-7 (FP64) / 1e-4 (mixed) relative."""
import numpy as np
import pytest

import oracle
import synth
from simhelp import deformed, dev, host, make_sim

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _prob(kind, muscle):
    p = synth.make_config1() if kind == "c1" else synth.make_small3d(6, 4, 4, split=6, seed=23)
    p.muscle_model = muscle
    if muscle:
        p.a = 0.5 + 0.5 * p.a
    return p


@pytest.mark.parametrize("kind", ["c1", "3d"])
@pytest.mark.parametrize("log_mode", [0, 1])
@pytest.mark.parametrize("muscle", [0, 1])
@pytest.mark.parametrize("dt", [0.0, 1.0 / 30.0])
def test_material_vjp_per_element(kind, log_mode, muscle, dt):
    p = _prob(kind, muscle)
    p.log_mode, p.dt = log_mode, dt
    sim = make_sim(p, "fp64", tile_elems=24, muscle_model=muscle)
    m = oracle.make_model(p)
    x = deformed(p, 0.03, seed=11)
    lam = np.random.default_rng(12).standard_normal(x.shape)
    lam[p.fixed.astype(bool)] = 0.0
    got = sim.material_vjp(dev(x), dev(p.a), dev(lam))
    ref = m.material_vjp(x, lam, p.a)
    for g, r in zip(got, ref):
        assert np.abs(host(g) - r).max() <= TOL64 * np.abs(r).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_quasistatic_material_gradient(precision):
    p = synth.make_small3d(8, 4, 4, split=5, seed=31)
    sim = make_sim(p, precision, tile_elems=128, adjoint_rtol=1e-10 if precision == "fp64" else 1e-6)
    m = oracle.make_model(p)
    a = dev(p.a)
    x, st = sim.solve(a)
    assert st["status"] == 0, st
    gL = oracle.mean_loss_grad(host(x), p.target)
    lam, _ = sim.adjoint(x, a, dev(gL))
    got = [float(host(g).sum()) for g in sim.material_vjp(x, a, lam)]
    x_or, lam_or, _, _ = oracle.quasistatic_forward_backward(m, p.a, p.target, rtol=1e-10)
    ref = [float(r.sum()) for r in m.material_vjp(x_or, lam_or, p.a)]
    tol = 1e-7 if precision == "fp64" else 1e-4
    for g, r in zip(got, ref):
        assert abs(g - r) <= tol * abs(r), (g, r)


def test_batch_per_mesh_material_gradients():
    """Batched rollouts of meshes with different mu: per-mesh dL/dmu,
    dL/dlambda, dL/dk over the whole rollout vs the oracle's BPTT."""
    import torch

    from paper_2102_05791_gb300.api import Batch
    probs = []
    for i, (nx, ny, mu) in enumerate([(4, 2, 1e4), (7, 3, 7e3), (5, 2, 1.6e4)]):
        p = synth.make_small2d(nx, ny, fix_bottom=False, seed=70 + i)
        p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
        p.mu, p.lam = mu, 4.0 * mu
        probs.append(p)
    b = Batch(probs, adjoint_rtol=1e-8)
    rng = np.random.default_rng(73)
    nT = 3
    a_seq = rng.uniform(0.0, 1.0, size=(nT, b.E))
    x0 = np.concatenate([p.X for p in probs])
    v0 = 0.1 * rng.standard_normal(x0.shape)
    xbT = rng.standard_normal(x0.shape)
    vbT = 0.01 * rng.standard_normal(x0.shape)
    out = b.rollout(dev(x0), dev(v0), dev(a_seq), dev(xbT), dev(vbT), material_grad=True)
    torch.cuda.synchronize()
    assert (host(out[5])[:, 0] == 0).all()
    mg = host(out[6])
    vo, eo = b.vert_offsets, b.elem_offsets
    for i, p in enumerate(probs):
        m = oracle.make_model(p)
        vs_, ve_ = vo[i], vo[i + 1]
        a_i = a_seq[:, eo[i]:eo[i + 1]]
        xs, vs = oracle.rollout(m, x0[vs_:ve_], v0[vs_:ve_], a_i, rtol=1e-10)
        _, _, _, mat = oracle.rollout_backward(m, xs, vs, a_i, xbT[vs_:ve_], vbT[vs_:ve_], material=True)
        assert np.abs(mg[i] - mat).max() <= 1e-4 * np.abs(mat).max(), (i, mg[i], mat)
    b.close()
