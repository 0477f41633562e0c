"""The stored oracle solutions (tests/golden/*_oracle.npz) against the oracle's
own definitions, on the CPU.

The large 3D body at 1/8 size and the 2 x 1 x 1 box of config 3: the stored state satisfies the Newton
tolerance it was solved to (|grad E(x*)| <= 1e-10 |grad E(X)|, Eq.
x1-quasistatic-argmin), the stored lambda solves H lambda = dL/dx to within
ten times the adjoint CG tolerance (CG stops on its recurred residual), and
the stored dL/da is the parameter VJP at (x*, lambda) (Eq. dLda-re-ordered).  The dynamics files carry the shapes, tolerances and
seeds the GPU comparisons rely on.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name", ["c5_eighth", "c3"])
def test_quasistatic_solution_is_the_oracles(name):
    g = np.load(os.path.join(GOLDEN, f"{name}_oracle.npz"))
    p = synth.make_config5(2) if name == "c5_eighth" else synth.make_config3()
    assert int(g["seed"]) == synth.BASE_SEED + (5 if name == "c5_eighth" else 3)
    m = oracle.make_model(p)
    x = p.X + g["u_star"]
    g0 = np.linalg.norm(m.grad(p.X, p.a))
    assert np.linalg.norm(m.grad(x, p.a)) <= 1.01 * float(g["newton_rtol"]) * g0
    b = oracle.mean_loss_grad(x, p.target)
    b[p.fixed.astype(bool)] = 0.0
    lam = g["lam"]
    # CG stops on its recurred residual; the true residual may be a few times larger
    assert np.linalg.norm(m.hvp(x, p.a, lam) - b) <= 10.0 * float(g["adjoint_rtol"]) * np.linalg.norm(b)
    # x* is stored as a displacement, so X + u* may differ from x* in the last bit
    ref = g["dLda"]
    assert np.abs(m.param_vjp(x, lam, p.a) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_dynamics_solutions_have_the_workload_shapes():
    c2 = np.load(os.path.join(GOLDEN, "c2_bptt_oracle.npz"))
    p = synth.make_config2()
    assert int(c2["seed"]) == synth.BASE_SEED + 2
    assert c2["g_groups"].shape == (200, p.extra["n_groups"])
    assert c2["xT"].shape == p.X.shape and np.isfinite(c2["xT"]).all()
    assert np.isfinite(c2["g_groups"]).all() and np.abs(c2["g_groups"]).max() > 0.0
    c4 = np.load(os.path.join(GOLDEN, "c4_bodies_oracle.npz"))
    probs = synth.make_config4(1024, int(c4["n_steps"]))
    sizes = np.array([q.n_elem for q in probs])
    order = np.argsort(sizes, kind="stable")
    for k, (i, q) in enumerate(zip(c4["bodies"], c4["quantiles"])):
        assert i == order[int(q * len(order))]
        assert c4[f"abar_{k}"].shape == (int(c4["n_steps"]), probs[i].n_elem)
        assert c4[f"xT_{k}"].shape == probs[i].X.shape
        assert np.isfinite(c4[f"abar_{k}"]).all()


@pytest.mark.parametrize("name", ["c5_eighth_oracle.npz", "c3_oracle.npz", "c2_bptt_oracle.npz",
                                  "c4_bodies_oracle.npz"])
def test_solution_files_record_their_tolerances(name):
    g = np.load(os.path.join(GOLDEN, name))
    assert "wall_s" in g and float(g["wall_s"]) > 0.0
    assert any(k in g for k in ("rtol", "newton_rtol"))
