"""Fault handling on the GPU, with every fault made on the host side.

* Non-finite inputs (a NaN position, velocity, activation or adjoint
  right-hand side) to the single-mesh solvers and to the batched solver end
  with SIM_ENAN; a NaN in one body of a batch leaves the other bodies'
  results as they are without it.
* A deliberately indefinite start (the oracle's dense Hessian there has a
  negative eigenvalue) ends in a minimum: CG's non-positive-curvature exit
  falls back to steepest descent, and the result satisfies the Newton
  tolerance with a positive definite Hessian (the oracle's Cholesky).
* A CG cap of one iteration gives a defined status and iteration counts.
* The bounded bulk-copy wait of the HVP tile kernel: with its first wait's
  poll limit set to zero the kernel gives up, lets its copies land, and the
  solve returns SIM_ECUDA with the "gave up waiting" message; with the limit
  restored the same handle solves again, bit for bit like a fresh handle.
No GPU is faulted or hung: the "timeout" is a wait limit the host sets.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from simhelp import dev, host, make_sim

pytestmark = pytest.mark.gpu

SIM_ECUDA, SIM_ENAN = -2, -6


def _nan_at(x, i, c=0):
    y = np.array(x, dtype=np.float64, copy=True)
    y[i, c] = np.nan
    return y


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_quasistatic_nan_inputs(precision):
    from paper_2102_05791_gb300.api import SimError
    p = synth.make_config1()
    sim = make_sim(p, precision)
    free = int(np.nonzero(p.fixed == 0)[0][5])
    a = dev(p.a)
    _, st = sim.solve(a, x_init=dev(_nan_at(p.X, free)), check=False)
    assert st["status"] == SIM_ENAN, st
    a_nan = p.a.copy()
    a_nan[7] = np.nan
    _, st = sim.solve(dev(a_nan), check=False)
    assert st["status"] == SIM_ENAN, st
    # the handle still works, and a NaN adjoint right-hand side is reported too
    x, st = sim.solve(a)
    assert st["status"] == 0, st
    with pytest.raises(SimError) as ei:
        sim.adjoint(x, a, dev(_nan_at(np.zeros_like(p.X), free, 1)))
    assert ei.value.code == SIM_ENAN
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("which", ["x0", "v0", "a"])
def test_step_nan_inputs(which, precision):
    from paper_2102_05791_gb300.api import SimError
    p = synth.make_small2d(6, 3, fix_bottom=False, seed=41)
    p.k_contact, p.dt = 1e6, 1.0 / 30.0
    sim = make_sim(p, precision, tile_elems=16)
    x0, v0, a = p.X.copy(), np.zeros_like(p.X), p.a.copy()
    if which == "x0":
        x0 = _nan_at(x0, 3)
    elif which == "v0":
        v0 = _nan_at(v0, 4, 1)
    else:
        a[2] = np.nan
    with pytest.raises(SimError) as ei:
        sim.step(dev(x0), dev(v0), dev(a))
    assert ei.value.code == SIM_ENAN
    sim.close()


def test_batch_nan_in_one_body():
    from paper_2102_05791_gb300.api import Batch
    probs = []
    for i, (nx, ny) in enumerate([(4, 2), (6, 3), (5, 3)]):
        p = synth.make_small2d(nx, ny, fix_bottom=False, seed=140 + i)
        p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
        probs.append(p)
    b = Batch(probs, adjoint_rtol=1e-8)
    rng = np.random.default_rng(141)
    a_seq = rng.uniform(0.0, 1.0, size=(3, b.E))
    x0 = np.concatenate([p.X for p in probs])
    v0 = 0.1 * rng.standard_normal(x0.shape)
    xbT = rng.standard_normal(x0.shape)
    zero = dev(np.zeros_like(x0))
    clean = b.rollout(dev(x0), dev(v0), dev(a_seq), dev(xbT), zero)
    torch.cuda.synchronize()
    assert (host(clean[5])[:, 0] == 0).all()
    vo, eo = b.vert_offsets, b.elem_offsets
    for kind in ("a", "x0"):
        a_bad, x_bad = a_seq.copy(), x0.copy()
        if kind == "a":
            a_bad[1, eo[1] + 2] = np.nan
        else:
            x_bad[vo[1] + 3, 0] = np.nan
        out = b.rollout(dev(x_bad), dev(v0), dev(a_bad), dev(xbT), zero)
        torch.cuda.synchronize()
        ms = host(out[5])
        assert ms[1, 0] == SIM_ENAN, (kind, ms)
        assert ms[0, 0] == 0 and ms[2, 0] == 0, (kind, ms)
        for i in (0, 2):  # the other bodies are computed exactly as before
            assert torch.equal(out[0][:, vo[i]:vo[i + 1]], clean[0][:, vo[i]:vo[i + 1]])
            assert torch.equal(out[2][:, eo[i]:eo[i + 1]], clean[2][:, eo[i]:eo[i + 1]])
    b.close()


def _indefinite_start(p, m):
    """Rest shape compressed to 55 % along x towards its left edge, plus noise
    (seed 0), pinned vertices at rest: J stays positive, H is indefinite."""
    X = p.X
    x = X.copy()
    x[:, 0] = X[:, 0].min() + 0.55 * (X[:, 0] - X[:, 0].min())
    x += 0.05 * np.random.default_rng(0).standard_normal(X.shape)
    fx = p.fixed.astype(bool)
    x[fx] = X[fx]
    return x


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_indefinite_start_reaches_a_minimum(precision):
    p = synth.make_small2d(4, 2, seed=7)
    m = oracle.make_model(p)
    free = m.free_mask()
    x_init = _indefinite_start(p, m)
    assert m.min_J(x_init) > 0.0
    H0 = m.dense_hessian(x_init, p.a)[np.ix_(free, free)]
    assert np.linalg.eigvalsh(0.5 * (H0 + H0.T))[0] < 0.0  # the start is indefinite
    sim = make_sim(p, precision, tile_elems=16)
    x, st = sim.solve(dev(p.a), x_init=dev(x_init))
    assert st["status"] == 0, st
    xg = host(x)
    g_init = np.linalg.norm(m.grad(x_init, p.a))
    assert np.linalg.norm(m.grad(xg, p.a)) <= 1.01e-8 * g_init
    H = m.dense_hessian(xg, p.a)[np.ix_(free, free)]
    np.linalg.cholesky(0.5 * (H + H.T))  # a minimum: positive definite
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cg_cap_of_one_iteration(precision):
    p = synth.make_config1()
    sim = make_sim(p, precision, max_cg=1, max_newton=400)
    x, st = sim.solve(dev(p.a), check=False)
    assert st["status"] in (0, -4), st  # converged, or the Newton cap
    assert st["cg_iters_total"] <= st["newton_iters"]
    if st["status"] == 0:
        m = oracle.make_model(p)
        g0 = np.linalg.norm(m.grad(p.X, p.a))
        assert np.linalg.norm(m.grad(host(x), p.a)) <= 1.01e-8 * g0
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bulk_copy_wait_gives_up_and_the_handle_recovers(precision):
    from paper_2102_05791_gb300.api import SimError
    p = synth.make_small3d(4, 3, 3, split=6, seed=61)
    a = dev(p.a)
    ref = make_sim(p, precision, tile_elems=32)
    x_ref, st_ref = ref.solve(a)
    assert st_ref["status"] == 0
    sim = make_sim(p, precision, tile_elems=32)
    sim.set_wait_limit(0)
    with pytest.raises(SimError) as ei:
        sim.solve(a)
    assert ei.value.code == SIM_ECUDA
    assert "gave up waiting" in str(ei.value)
    sim.set_wait_limit(-1)
    x, st = sim.solve(a)
    assert st["status"] == 0, st
    assert torch.equal(x, x_ref)  # same handle, clean state: bit-identical to a fresh one
    ref.close()
    sim.close()
