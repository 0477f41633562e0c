"""The tile-shape autotuner: picks one of its candidates by the time per CG
iteration of a short solve, caches the choice, and a cached choice is reused
without measuring."""
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_and_caches(tmp_path, monkeypatch):
    from paper_2102_05791_gb300 import autotune
    from paper_2102_05791_gb300.api import Simulator
    monkeypatch.setenv("SOFTSIM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    p = synth.make_small3d(8, 4, 4, split=6, seed=80)
    mat = dict(mu=p.mu, lam=p.lam, k_muscle=p.k_muscle, density=p.density, gravity=p.gravity)
    cands = [(96, 128), (192, 128)]
    best = autotune.best_tile_shape(p.X, p.T, p.fixed, p.fiber, candidates=cands, **mat)
    assert best in cands
    monkeypatch.setattr(autotune, "measure", lambda *a, **k: pytest.fail("cache not used"))
    assert autotune.best_tile_shape(p.X, p.T, p.fixed, p.fiber, candidates=cands, **mat) == best
    sim = Simulator(p.X, p.T, p.fixed, p.fiber, tile_elems="auto", device="cuda:0", **mat)
    assert sim.tile_shape == best
    sim.close()
