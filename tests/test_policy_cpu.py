"""CPU checks of the policy demo's plumbing (no simulator): output range
and shape, translation invariance of the state features, and an episode
driven through a stand-in step function."""
import torch

from paper_2102_05791_gb300 import policy as pol


def test_policy_output_range_and_translation_invariance():
    torch.manual_seed(0)
    n, d, g = 30, 2, 8
    P = pol.MusclePolicy(n, d, g, a_min=0.25, a_max=0.9).double()
    X = torch.randn(n, d, dtype=torch.float64)
    x = X + 0.01 * torch.randn(n, d, dtype=torch.float64)
    v = torch.randn(n, d, dtype=torch.float64)
    a = P(x, v, X)
    assert a.shape == (g,)
    assert bool((a >= 0.25).all()) and bool((a <= 0.9).all())
    shift = torch.tensor([3.0, 0.5], dtype=torch.float64)
    assert torch.allclose(P(x + shift, v, X), a, rtol=0, atol=1e-12)


def test_episode_chains_steps_and_backpropagates(monkeypatch):
    """With a stand-in step x1 = x0 + dt v1, v1 = v0 + mean(a), the reward is
    differentiable in the policy weights through every step."""
    class FakeStep:
        @staticmethod
        def apply(sim, x0, v0, a):
            v1 = v0 + a.mean()
            return x0 + 0.1 * v1, v1

    monkeypatch.setattr(pol, "BEStep", FakeStep)
    torch.manual_seed(1)
    n, d, g = 12, 2, 3
    P = pol.MusclePolicy(n, d, g).double()
    X = torch.randn(n, d, dtype=torch.float64)
    group = torch.randint(0, g, (20,))
    reward, xT = pol.episode(None, P, X, group, 3)
    assert xT.shape == X.shape
    reward.backward()
    assert all(q.grad is not None and torch.isfinite(q.grad).all() for q in P.parameters())
    assert any(float(q.grad.abs().sum()) > 0 for q in P.parameters())
