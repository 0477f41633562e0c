"""Policy-in-the-loop BPTT (Sec. 5 usage): a 32-unit ReLU policy drives the
walker's muscle groups through backward-Euler steps; the reward gradient
reaches the policy weights through every step's adjoint.

Checked: the autograd gradient of the episode reward against central finite
differences along a random weight direction (FP64 handle, tight solves,
relative error <= 1e-4), and that a few Adam steps raise the reward."""
import numpy as np
import pytest
import torch

import synth
from simhelp import make_sim

pytestmark = pytest.mark.gpu


def _setup(precision, n_steps, **kw):
    from paper_2102_05791_gb300.policy import MusclePolicy
    p = synth.make_config2(n_steps=n_steps, nx=16, ny=8)
    sim = make_sim(p, precision, k_friction=2e3, **kw)
    X = torch.from_numpy(p.X).cuda()
    group = torch.from_numpy(p.extra["group"].astype(np.int64)).cuda()
    torch.manual_seed(3)
    policy = MusclePolicy(p.n_vert, p.dim, p.extra["n_groups"]).double().cuda()
    return p, sim, X, group, policy


def test_policy_gradient_matches_fd():
    from paper_2102_05791_gb300.policy import episode
    n_steps = 4
    p, sim, X, group, policy = _setup("fp64", n_steps, newton_rtol=1e-12, adjoint_rtol=1e-12)
    reward, _ = episode(sim, policy, X, group, n_steps)
    params = list(policy.parameters())
    grads = torch.autograd.grad(reward, params)
    gen = torch.Generator(device="cpu").manual_seed(4)
    dirs = [torch.randn(q.shape, generator=gen, dtype=torch.float64).cuda() for q in params]
    norm = float(torch.sqrt(sum((d * d).sum() for d in dirs)))
    dirs = [d / norm for d in dirs]  # unit direction in weight space
    an = sum(float((g * d).sum()) for g, d in zip(grads, dirs))

    def central(eps):
        vals = []
        with torch.no_grad():
            for sgn in (1.0, -1.0):
                for q, d in zip(params, dirs):
                    q.add_(sgn * eps * d)
                r, _ = episode(sim, policy, X, group, n_steps)
                vals.append(float(r))
                for q, d in zip(params, dirs):
                    q.sub_(sgn * eps * d)
        return (vals[0] - vals[1]) / (2 * eps)

    # Richardson extrapolation of the central difference: O(eps^4) truncation
    fd = (4.0 * central(1e-4) - central(2e-4)) / 3.0
    assert abs(an) > 0.0
    assert abs(fd - an) <= 1e-4 * abs(an), (fd, an)


def test_adam_raises_the_reward():
    from paper_2102_05791_gb300.policy import train
    n_steps = 10
    p, sim, X, group, policy = _setup("mixed", n_steps, adjoint_rtol=1e-8)
    rewards = train(sim, policy, X, group, n_steps, iters=8, lr=1e-2)
    assert all(np.isfinite(rewards))
    assert max(rewards[1:]) > rewards[0], rewards
