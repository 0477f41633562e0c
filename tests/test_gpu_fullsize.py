"""Parity at the benchmark's full sizes, in the benchmark's launch configuration.

* The large 3D body (128x64x64 hexes x 6 tets: 3,145,728 tets, 545,025
  vertices), handle built as bench.py builds it (mixed precision, autotuned
  tile shape): the FP64 gradient and the FP32 HVP at a deformed state against
  the oracle's full passes; then the benchmark's forward + adjoint + VJP, checked
  by properties the oracle evaluates at the GPU's answer (gradient residual,
  adjoint residual, and the VJP at the GPU's state and adjoint).
* The 1,024-body batch (2D, 200-8,000 triangles each, 60 backward-Euler steps,
  forward + BPTT in one launch, adjoint tolerance 1e-8) as bench.py runs it: three bodies spread over
  the size range against the oracle's stored rollout and BPTT.

Tolerances: as in the other parity tests (FP64 kernels 1e-12 of the
contribution scale, FP32 HVP 1e-5 of the largest entry, gradient residual
1.01e-8 of |g0|, adjoint residual 1e-4 with adjoint_rtol 1e-6); for the 60-step
rollouts states within 1e-5 of the displacement scale and gradients within
1e-4 relative L2.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from simhelp import deformed, dev, host, make_sim

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def test_large_3d_body_full_size():
    p = synth.make_config5()
    sim = make_sim(p, "mixed", tile_elems="auto")
    m = oracle.make_model(p)
    a = dev(p.a)
    # element kernels at a deformed, non-equilibrium state
    x = deformed(p, 0.005, seed=15)
    E, g = sim.energy_grad(dev(x), a)
    E_or, S_or = m.energy(x, p.a, with_abs=True)
    g_or, scale = m.grad(x, p.a, with_scale=True)
    assert abs(float(E) - E_or) <= TOL64 * S_or
    assert np.abs(host(g) - g_or).max() <= TOL64 * scale.max()
    v = np.random.default_rng(16).standard_normal(x.shape).astype(np.float32).astype(np.float64)
    Hv = host(sim.hvp(dev(x), a, dev(v, sim.vec_dtype))).astype(np.float64)
    Hv_or = m.hvp(x, p.a, v)
    assert np.abs(Hv - Hv_or).max() <= TOL32 * np.abs(Hv_or).max()
    # the benchmark's step: forward solve, adjoint, VJP
    xs, st = sim.solve(a)
    assert st["status"] == 0, st
    xg = host(xs)
    g0 = np.linalg.norm(m.grad(p.X, p.a))
    assert np.linalg.norm(m.grad(xg, p.a)) <= 1.01e-8 * g0
    gL = oracle.mean_loss_grad(xg, p.target)
    lam, st_a = sim.adjoint(xs, a, dev(gL))
    assert st_a["status"] == 0, st_a
    lg = host(lam)
    b = gL.copy()
    b[p.fixed.astype(bool)] = 0.0
    assert np.linalg.norm(m.hvp(xg, p.a, lg) - b) <= 1e-4 * np.linalg.norm(b)
    dLda = host(sim.param_vjp(xs, a, lam))
    ref = m.param_vjp(xg, lg, p.a)
    assert np.abs(dLda - ref).max() <= TOL64 * np.abs(ref).max()


def test_thousand_body_batch_full_size():
    from paper_2102_05791_gb300.api import Batch
    n_steps = 60
    probs = synth.make_config4(1024, n_steps)
    x0 = np.concatenate([p.X for p in probs])
    a_seq = np.concatenate([p.extra["a_seq"] for p in probs], axis=1)
    xbT = np.zeros_like(x0)
    off = 0
    for p in probs:
        xbT[off:off + p.n_vert, 0] = 1.0 / p.n_vert
        off += p.n_vert
    b = Batch(probs, newton_rtol=1e-8, adjoint_rtol=1e-8, threads="auto")
    sx, sv, abar, xb0, vb0, ms = b.rollout(dev(x0), dev(np.zeros_like(x0)), dev(a_seq), dev(xbT),
                                           dev(np.zeros_like(x0)))
    torch.cuda.synchronize()
    ms = host(ms)
    assert (ms[:, 0] == 0).all(), np.nonzero(ms[:, 0])
    sx, abar, vb0 = host(sx), host(abar), host(vb0)
    vo, eo = b.vert_offsets, b.elem_offsets
    order = np.argsort([p.n_elem for p in probs])
    for i in (order[0], order[len(order) // 2], order[int(0.8 * len(order))]):
        p = probs[i]
        m = oracle.make_model(p)
        vs_, ve_ = vo[i], vo[i + 1]
        a_i = a_seq[:, eo[i]:eo[i + 1]]
        xs, vs = oracle.rollout(m, p.X.copy(), np.zeros_like(p.X), a_i, rtol=1e-10)
        assert np.abs(sx[-1, vs_:ve_] - xs[-1]).max() <= 1e-5 * np.abs(xs[-1] - xs[0]).max(), p.name
        _, vb, ab = oracle.rollout_backward(m, xs, vs, a_i, xbT[vs_:ve_], np.zeros_like(p.X))
        assert np.linalg.norm(abar[:, eo[i]:eo[i + 1]] - ab) <= 1e-4 * np.linalg.norm(ab), p.name
        assert np.linalg.norm(vb0[vs_:ve_] - vb) <= 1e-4 * np.linalg.norm(vb), p.name
    b.close()


def test_cg_inner_product_error_against_fp64():
    """The mixed CG loop's p.Ap on the large 3D body in the benchmark's launch
    configuration: FP32 element quadratic forms, plain FP32 sums within each
    384-tet tile, compensated FP32 sums over the 8,192 tiles.  Against the
    FP64 v.(H v) of the oracle (which also carries the FP32 HVP's own
    rounding), and against the FP64 dot of the kernel's own FP32 H v (the
    summation alone); both within 1e-5 relative."""
    p = synth.make_config5()
    sim = make_sim(p, "mixed", tile_elems="auto")
    m = oracle.make_model(p)
    x = deformed(p, 0.005, seed=15)
    v = np.random.default_rng(17).standard_normal(x.shape).astype(np.float32).astype(np.float64)
    Hv, q = sim.hvp_dot(dev(x), dev(p.a), dev(v, sim.vec_dtype))
    q64 = float(np.dot(v.ravel(), m.hvp(x, p.a, v).ravel()))
    assert q64 > 0.0
    assert abs(q - q64) <= 1e-5 * q64, (q, q64)
    q_own = float(np.dot(v.ravel(), host(Hv).astype(np.float64).ravel()))
    assert abs(q - q_own) <= 1e-5 * abs(q_own), (q, q_own)
