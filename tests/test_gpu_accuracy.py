"""GPU results of the benchmark workloads against the oracle's own solutions.

The stored solutions (tests/golden/*_oracle.npz) are written by
tests/golden/make_oracle_solutions.py, which calls only the FP64 oracle:

* the large 3D body at 1/8 size (64 x 32 x 32 hexes x 6 tets, 393,216 tets)
  and the 2 x 1 x 1 box of config 3 (40,960 tets): the quasistatic state x*
  (Eq. x1-quasistatic-argmin), the adjoint lambda and dL/da (Eq.
  dLda-re-ordered) of L = 1/2 |mean(x) - target|^2, compared with the GPU's
  forward solve, adjoint and parameter VJP in both precisions, in the
  benchmark's launch configuration (autotuned tiles for the mixed path);
* the 64 x 32 walker, 200 backward-Euler steps (Eq. opt-be) with BPTT
  (Sec. 4): the final state and dL/d(a_groups), against the checkpointed GPU
  rollout and its backward as the benchmark runs them (adjoints to 1e-8: at
  1e-6 the 200-step group gradient is off by 1.4e-3 relative);
* three bodies of the 1,024-body batch: the 60-step BPTT gradients of each
  body against the batched persistent solver.

Bars: states within 1e-5 of the displacement scale; gradients within 1e-4
relative L2 for the mixed path and 1e-7 for the FP64 path.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from simhelp import dev, host, make_sim

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("name", ["c5_eighth", "c3"])
def test_quasistatic_workload_matches_oracle_solution(name, precision):
    g = np.load(os.path.join(GOLDEN, f"{name}_oracle.npz"))
    p = synth.make_config5(2) if name == "c5_eighth" else synth.make_config3()
    kw = {"tile_elems": "auto"} if precision == "mixed" else {"adjoint_rtol": 1e-10}
    sim = make_sim(p, precision, **kw)
    a = dev(p.a)
    xs, st = sim.solve(a)
    assert st["status"] == 0, st
    xg = host(xs)
    u_or = g["u_star"]
    assert np.abs((xg - p.X) - u_or).max() <= 1e-5 * np.abs(u_or).max()
    lam, sta = sim.adjoint(xs, a, dev(oracle.mean_loss_grad(xg, p.target)))
    assert sta["status"] == 0, sta
    dLda = host(sim.param_vjp(xs, a, lam))
    tol = 1e-4 if precision == "mixed" else 1e-7
    assert _rel(host(lam), g["lam"]) <= tol
    assert _rel(dLda, g["dLda"]) <= tol
    sim.close()


def test_walker_bptt_matches_oracle_solution():
    g = np.load(os.path.join(GOLDEN, "c2_bptt_oracle.npz"))
    p = synth.make_config2()
    group = torch.from_numpy(p.extra["group"].astype(np.int64)).cuda()
    sim = make_sim(p, "mixed", tile_elems="auto", adjoint_rtol=1e-8)
    a_groups = dev(p.extra["a_groups"])
    a_seq = a_groups[:, group].contiguous()
    x0 = dev(p.X)
    xT, vT, ck, st = sim.rollout(x0, torch.zeros_like(x0), a_seq, ckpt_every=20)
    assert st["status"] == 0, st
    scale = np.abs(g["xT"] - p.X).max()
    assert np.abs(host(xT) - g["xT"]).max() <= 1e-5 * scale
    xbT = torch.zeros_like(x0)
    xbT[:, 0] = 1.0 / p.n_vert
    _, vb0, ab, _ = sim.rollout_backward(a_seq, ck, 20, xbT, torch.zeros_like(x0))
    g_groups = host(torch.zeros_like(a_groups).index_add_(1, group, ab))
    assert _rel(g_groups, g["g_groups"]) <= 1e-4
    assert _rel(host(vb0), g["vbar0"]) <= 1e-4
    sim.close()


def test_batch_bodies_match_oracle_solutions():
    from paper_2102_05791_gb300.api import Batch
    g = np.load(os.path.join(GOLDEN, "c4_bodies_oracle.npz"))
    n_steps = int(g["n_steps"])
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
    assert (host(ms)[:, 0] == 0).all()
    sx, abar, vb0 = host(sx), host(abar), host(vb0)
    vo, eo = b.vert_offsets, b.elem_offsets
    for k, i in enumerate(g["bodies"]):
        p = probs[i]
        scale = np.abs(g[f"xT_{k}"] - p.X).max()
        assert np.abs(sx[-1, vo[i]:vo[i + 1]] - g[f"xT_{k}"]).max() <= 1e-5 * scale, p.name
        assert _rel(abar[:, eo[i]:eo[i + 1]], g[f"abar_{k}"]) <= 1e-4, p.name
        assert _rel(vb0[vo[i]:vo[i + 1]], g[f"vbar0_{k}"]) <= 1e-4, p.name
    b.close()
