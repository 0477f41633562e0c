"""Batched persistent rollouts (many meshes, one launch) vs the oracle's
per-mesh backward-Euler rollout and BPTT (Eq. opt-be, Eq. dLda-re-ordered).

Tolerances: states within 1e-6 of the displacement scale (both converge to
|g| <= 1e-8 |g0| per step); gradients within 1e-4 relative L2 (mixed
precision with FP64-refined adjoints)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from simhelp import dev, host

pytestmark = pytest.mark.gpu


def _meshes():
    out = []
    for i, (nx, ny, mu) in enumerate([(4, 2, 1e4), (7, 3, 7e3), (5, 2, 1.6e4), (9, 4, 5.5e3)]):
        p = synth.make_small2d(nx, ny, fix_bottom=False, seed=60 + i)
        p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
        p.mu, p.lam = mu, 4.0 * mu
        out.append(p)
    return out


def test_batch_rollout_matches_oracle_and_is_deterministic():
    from paper_2102_05791_gb300.api import Batch
    probs = _meshes()
    b = Batch(probs, adjoint_rtol=1e-8)
    rng = np.random.default_rng(70)
    nT = 3
    E = b.E
    a_seq = rng.uniform(0.0, 1.0, size=(nT, E))
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
        scale = max(np.abs(xs[-1] - xs[0]).max(), 1e-6)
        assert np.abs(sx[-1, vs_:ve_] - xs[-1]).max() <= 1e-6 * scale
        xb, vb, ab = oracle.rollout_backward(m, xs, vs, a_i, xbT[vs_:ve_], vbT[vs_:ve_])
        assert np.linalg.norm(abar[:, es_:ee_] - ab) <= 1e-4 * np.linalg.norm(ab)
        assert np.linalg.norm(vb0[vs_:ve_] - vb) <= 1e-4 * np.linalg.norm(vb)
        assert np.linalg.norm(xb0[vs_:ve_] - xb) <= 1e-4 * np.linalg.norm(xb)
    # same inputs, second launch (graph replay): bit-identical
    sx2, sv2, abar2, xb02, vb02, ms2 = b.rollout(dev(x0), dev(v0), dev(a_seq), dev(xbT), dev(vbT))
    torch.cuda.synchronize()
    assert np.array_equal(host(abar2), abar)
    assert np.array_equal(host(sx2), sx)
    b.close()


def test_batch_rejects_mixed_dims_and_materials():
    from paper_2102_05791_gb300.api import Batch, SimError
    probs = _meshes()[:2]
    probs[1].k_muscle = 1.0
    with pytest.raises(SimError):
        Batch(probs)


@pytest.mark.parametrize("threads", [128, 512])
def test_batch_block_sizes_agree(threads):
    """Every block size the autotuner may pick gives the 256-thread result
    within the parity tolerances (the fixed-order sums differ in grouping)."""
    from paper_2102_05791_gb300.api import Batch
    probs = _meshes()
    rng = np.random.default_rng(71)
    nT = 2
    x0 = np.concatenate([p.X for p in probs])
    v0 = 0.1 * rng.standard_normal(x0.shape)
    xbT = rng.standard_normal(x0.shape)
    outs = {}
    for th in (256, threads):
        b = Batch(probs, adjoint_rtol=1e-8, threads=th)
        a_seq = rng.uniform(0.0, 1.0, size=(nT, b.E)) if th == 256 else a_seq
        sx, sv, abar, xb0, vb0, ms = b.rollout(dev(x0), dev(v0), dev(a_seq), dev(xbT), dev(np.zeros_like(x0)))
        torch.cuda.synchronize()
        assert (host(ms)[:, 0] == 0).all()
        outs[th] = (host(sx), host(abar))
        assert b.threads == th
        b.close()
    (s1, g1), (s2, g2) = outs[256], outs[threads]
    assert np.abs(s1[-1] - s2[-1]).max() <= 1e-6 * np.abs(s1[-1] - s1[0]).max()
    assert np.linalg.norm(g1 - g2) <= 1e-4 * np.linalg.norm(g1)


def test_batch_autotuner_picks_a_candidate(tmp_path, monkeypatch):
    from paper_2102_05791_gb300 import autotune
    from paper_2102_05791_gb300.api import Batch
    monkeypatch.setenv("SOFTSIM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    b = Batch(_meshes(), threads="auto")
    assert b.threads in autotune.BATCH_CANDIDATES
    b.close()
    # second time from the cache
    assert autotune.best_batch_threads(_meshes()) == b.threads


def test_batch_rejects_unsupported_block_size():
    from paper_2102_05791_gb300.api import Batch, SimError
    with pytest.raises(SimError):
        Batch(_meshes(), threads=96)


def _check_batch_against_oracle(probs, a_lo, a_hi, seed, threads=256, tol_g=1e-4):
    from paper_2102_05791_gb300.api import Batch
    b = Batch(probs, adjoint_rtol=1e-8, threads=threads)
    rng = np.random.default_rng(seed)
    nT = 3
    a_seq = rng.uniform(a_lo, a_hi, size=(nT, b.E))
    x0 = np.concatenate([p.X for p in probs])
    v0 = 0.1 * rng.standard_normal(x0.shape)
    xbT = rng.standard_normal(x0.shape)
    vbT = 0.01 * rng.standard_normal(x0.shape)
    sx, sv, abar, xb0, vb0, ms, mg = b.rollout(dev(x0), dev(v0), dev(a_seq), dev(xbT), dev(vbT),
                                               material_grad=True)
    torch.cuda.synchronize()
    ms = host(ms)
    assert (ms[:, 0] == 0).all(), ms
    sx, abar, xb0, vb0, mg = host(sx), host(abar), host(xb0), host(vb0), host(mg)
    vo, eo = b.vert_offsets, b.elem_offsets
    for i, p in enumerate(probs):
        m = oracle.make_model(p)
        vs_, ve_ = vo[i], vo[i + 1]
        a_i = a_seq[:, eo[i]:eo[i + 1]]
        xs, vs = oracle.rollout(m, x0[vs_:ve_], v0[vs_:ve_], a_i, rtol=1e-10)
        assert np.abs(sx[-1, vs_:ve_] - xs[-1]).max() <= 1e-6 * np.abs(xs[-1] - xs[0]).max()
        xb, vb, ab, mat = oracle.rollout_backward(m, xs, vs, a_i, xbT[vs_:ve_], vbT[vs_:ve_], material=True)
        assert np.linalg.norm(abar[:, eo[i]:eo[i + 1]] - ab) <= tol_g * np.linalg.norm(ab)
        assert np.linalg.norm(vb0[vs_:ve_] - vb) <= tol_g * np.linalg.norm(vb)
        assert np.linalg.norm(xb0[vs_:ve_] - xb) <= tol_g * np.linalg.norm(xb)
        assert np.abs(mg[i] - mat).max() <= tol_g * np.abs(mat).max()
    b.close()


@pytest.mark.parametrize("threads", [128, 512])
def test_batch_3d_tet_meshes(threads):
    """The 3D persistent kernel: uneven tet meshes with their own mu, forward
    + BPTT + material gradients against the oracle."""
    probs = []
    for i, (nx, ny, nz, split, mu) in enumerate([(2, 2, 2, 5, 1e4), (3, 2, 2, 6, 7e3), (2, 3, 2, 5, 1.5e4)]):
        p = synth.make_small3d(nx, ny, nz, split=split, fix_bottom=False, seed=100 + i)
        p.k_contact, p.contact_power, p.dt = 1e6, 3, 1.0 / 30.0
        p.mu, p.lam = mu, 4.0 * mu
        probs.append(p)
    _check_batch_against_oracle(probs, 0.0, 1.0, 101, threads=threads)


def test_batch_friction_with_spring_muscle():
    """Friction and the active-spring muscle together in the batched solver."""
    probs = []
    for i, (nx, ny) in enumerate([(4, 2), (6, 3)]):
        p = synth.make_small2d(nx, ny, fix_bottom=False, seed=110 + i)
        p.k_contact, p.contact_power, p.dt = 1e5, 2, 1.0 / 30.0
        p.k_friction, p.eps_friction = 2e3, 0.01
        p.muscle_model = 1
        probs.append(p)
    _check_batch_against_oracle(probs, 0.5, 1.0, 111)
