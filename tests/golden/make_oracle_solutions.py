#!/usr/bin/env python3
"""Writes the oracle's own solutions of the benchmark workloads to tests/golden/.

Every stored value comes from the FP64 CPU oracle (``oracle/``) on the seeded
inputs of ``synth``; nothing here touches the CUDA library.  The GPU tests and
the benchmark's accuracy report compare the GPU results with these files.

* ``c5_eighth_oracle.npz`` -- the large 3D body at 1/8 size (4 x 2 x 2 box,
  64 x 32 x 32 hexes x 6 tets: 70,785 vertices, 393,216 tets; seed 20210211 + 5):
  the quasistatic solve x* = argmin E(x, a) (Eq. x1-quasistatic-argmin) by the
  oracle's Newton-CG to |grad E| <= 1e-10 |grad E_0|, the adjoint
  lambda = H^-1 dL/dx (Eq. dLda-re-ordered) by CG to 1e-11 relative residual,
  and dL/da = -lambda^T d2E/dx da, for L = 1/2 |mean(x) - target|^2.
* ``c3_oracle.npz`` -- the 2 x 1 x 1 box (32 x 16 x 16 hexes x 5 tets: 9,537
  vertices, 40,960 tets; seed 20210211 + 3), the same three quantities as for
  the large body, at the same tolerances.
* ``c2_bptt_oracle.npz`` -- the 64 x 32 walker (2,145 vertices, 4,096 tris;
  seed 20210211 + 2), 200 backward-Euler steps (Eq. opt-be) at rtol 1e-10,
  then backpropagation through time (Sec. 4) of the horizontal displacement
  of the vertex mean, adjoints to 1e-12: the final state and dL/d(a_groups),
  the gradient with respect to the 8 groups' activations at every step.
* ``c4_bodies_oracle.npz`` -- three bodies of the 1,024-body batch (seed
  20210211 + 4): the smallest, the median and the 80th-percentile body by
  triangle count, 60 backward-Euler steps at rtol 1e-10, BPTT of each body's
  mean horizontal position (adjoints to 1e-12): final states, dL/dv_0 and
  dL/da per step and element.

Run from the repository root: ``python tests/golden/make_oracle_solutions.py``
(about ten minutes on three host cores; each workload runs in its own
process, each single-threaded).
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

C5_NEWTON_RTOL = 1e-10
C5_ADJ_RTOL = 1e-11
DYN_RTOL = 1e-10
DYN_ADJ_RTOL = 1e-12
C4_PICK_QUANTILES = (0.0, 0.5, 0.8)   # positions in the batch sorted by triangle count


def c4_pick(probs):
    order = np.argsort([p.n_elem for p in probs], kind="stable")
    return [int(order[int(q * len(order))]) if q < 1.0 else int(order[-1]) for q in C4_PICK_QUANTILES]


def _quasistatic(p, name, seed):
    import oracle
    m = oracle.make_model(p)
    t0 = time.perf_counter()
    x, st = m.newton(p.a, rtol=C5_NEWTON_RTOL)
    if st["status"] != oracle.OK:
        raise RuntimeError(f"oracle Newton status {st}")
    gL = oracle.mean_loss_grad(x, p.target)
    lam, it = m.adjoint(x, p.a, gL, rtol=C5_ADJ_RTOL)
    dLda = m.param_vjp(x, lam, p.a)
    wall = time.perf_counter() - t0
    np.savez_compressed(os.path.join(HERE, name), u_star=x - p.X, lam=lam, dLda=dLda,
                        newton_rtol=C5_NEWTON_RTOL, adjoint_rtol=C5_ADJ_RTOL, seed=seed,
                        newton_iters=st["newton_iters"], cg_iters=st["cg_iters_total"], adjoint_cg_iters=it,
                        res0=st["res0"], res_final=st["res_final"], wall_s=wall)
    return f"{name}: newton {st['newton_iters']} cg {st['cg_iters_total']} adjoint cg {it}, {wall:.0f} s"


def c3():
    import synth
    return _quasistatic(synth.make_config3(), "c3_oracle.npz", synth.BASE_SEED + 3)


def c5_eighth():
    import oracle
    import synth
    p = synth.make_config5(2)
    m = oracle.make_model(p)
    t0 = time.perf_counter()
    x, st = m.newton(p.a, rtol=C5_NEWTON_RTOL)
    if st["status"] != oracle.OK:
        raise RuntimeError(f"oracle Newton status {st}")
    gL = oracle.mean_loss_grad(x, p.target)
    lam, it = m.adjoint(x, p.a, gL, rtol=C5_ADJ_RTOL)
    dLda = m.param_vjp(x, lam, p.a)
    wall = time.perf_counter() - t0
    np.savez_compressed(os.path.join(HERE, "c5_eighth_oracle.npz"), u_star=x - p.X, lam=lam, dLda=dLda,
                        newton_rtol=C5_NEWTON_RTOL, adjoint_rtol=C5_ADJ_RTOL, seed=synth.BASE_SEED + 5,
                        newton_iters=st["newton_iters"], cg_iters=st["cg_iters_total"], adjoint_cg_iters=it,
                        res0=st["res0"], res_final=st["res_final"], wall_s=wall)
    return f"c5_eighth: newton {st['newton_iters']} cg {st['cg_iters_total']} adjoint cg {it}, {wall:.0f} s"


def c2_bptt():
    import oracle
    import synth
    p = synth.make_config2()
    m = oracle.make_model(p)
    group = p.extra["group"]
    a_seq = p.extra["a_groups"][:, group]
    x0, v0 = p.X.copy(), np.zeros_like(p.X)
    t0 = time.perf_counter()
    xs, vs = oracle.rollout(m, x0, v0, a_seq, rtol=DYN_RTOL)
    xbT = np.zeros_like(x0)
    xbT[:, 0] = 1.0 / p.n_vert
    _, vb0, ab = oracle.rollout_backward(m, xs, vs, a_seq, xbT, np.zeros_like(x0), adj_rtol=DYN_ADJ_RTOL)
    wall = time.perf_counter() - t0
    g_groups = np.stack([np.bincount(group, weights=ab[t], minlength=p.extra["n_groups"])
                         for t in range(len(a_seq))])
    np.savez_compressed(os.path.join(HERE, "c2_bptt_oracle.npz"), xT=xs[-1], vT=vs[-1], g_groups=g_groups,
                        vbar0=vb0, rtol=DYN_RTOL, adjoint_rtol=DYN_ADJ_RTOL, seed=synth.BASE_SEED + 2,
                        n_steps=len(a_seq), wall_s=wall)
    return f"c2_bptt: {len(a_seq)} steps, {wall:.0f} s"


def c4_bodies():
    import oracle
    import synth
    probs = synth.make_config4(1024, 60)
    out = {}
    t0 = time.perf_counter()
    pick = c4_pick(probs)
    for k, i in enumerate(pick):
        p = probs[i]
        m = oracle.make_model(p)
        a_i = p.extra["a_seq"]
        xs, vs = oracle.rollout(m, p.X.copy(), np.zeros_like(p.X), a_i, rtol=DYN_RTOL)
        xbT = np.zeros_like(p.X)
        xbT[:, 0] = 1.0 / p.n_vert
        _, vb, ab = oracle.rollout_backward(m, xs, vs, a_i, xbT, np.zeros_like(p.X), adj_rtol=DYN_ADJ_RTOL)
        out[f"xT_{k}"] = xs[-1]
        out[f"vbar0_{k}"] = vb
        out[f"abar_{k}"] = ab
    wall = time.perf_counter() - t0
    np.savez_compressed(os.path.join(HERE, "c4_bodies_oracle.npz"), bodies=np.array(pick),
                        quantiles=np.array(C4_PICK_QUANTILES), rtol=DYN_RTOL, adjoint_rtol=DYN_ADJ_RTOL,
                        seed=synth.BASE_SEED + 4, n_steps=60, wall_s=wall, **out)
    return f"c4_bodies: bodies {pick}, {wall:.0f} s"


def _run(name):
    return {"c5_eighth": c5_eighth, "c3": c3, "c2_bptt": c2_bptt, "c4_bodies": c4_bodies}[name]()


def main(argv):
    names = argv or ["c5_eighth", "c3", "c2_bptt", "c4_bodies"]
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for msg in pool.imap_unordered(_run, names):
            print(msg, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
