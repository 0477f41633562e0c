"""Policy-in-the-loop training through the differentiable simulator (Sec. 5).

A control policy maps the body's state (vertex positions and velocities) to
muscle activations at every backward-Euler step; an episode's reward is the
horizontal displacement of the body's vertex mean after n steps.  The reward's
gradient with respect to the policy weights flows back through every step
(backpropagation through time): each step is an ``api.BEStep``, whose backward
is the implicit-differentiation adjoint of the step (Eq. opt-be) computed by
this library's kernels, and the policy sees the state, so the gradient also
flows through the policy's inputs.

The paper's policies have one hidden layer of 32 ReLU units, take the
simulation state as input, output the fibers' actions, and are trained with
Adam at learning rate 1e-3; ``MusclePolicy`` and ``train`` build that network
and loop.  The network is plain PyTorch; the simulation is the part that runs
in this library.

    python -m paper_2102_05791_gb300.policy --iters 20      # 64 x 32 walker
"""
from __future__ import annotations

import argparse
import time

import torch

from .api import BEStep, Simulator


class MusclePolicy(torch.nn.Module):
    """state -> per-group activations in [a_min, a_max] (one hidden ReLU layer)."""

    def __init__(self, n_vert: int, dim: int, n_groups: int, hidden: int = 32, a_min: float = 0.2,
                 a_max: float = 1.0):
        super().__init__()
        self.a_min, self.a_max = float(a_min), float(a_max)
        self.net = torch.nn.Sequential(torch.nn.Linear(2 * n_vert * dim, hidden), torch.nn.ReLU(),
                                       torch.nn.Linear(hidden, n_groups))

    def forward(self, x, v, X):
        # shape relative to the centroid (invariant to where the body has walked) and velocities
        d = (x - x.mean(dim=0)) - (X - X.mean(dim=0))
        feat = torch.cat([d.reshape(-1), v.reshape(-1)])
        return self.a_min + (self.a_max - self.a_min) * torch.sigmoid(self.net(feat))


def episode(sim: Simulator, policy: MusclePolicy, X, group, n_steps: int, v0=None):
    """Roll out n_steps under the policy from rest; returns (reward, x_T).

    X: rest positions [n_vert, dim] (float64, on the simulator's device);
    group: element -> muscle group index [n_elem] (int64)."""
    x = X
    v = torch.zeros_like(X) if v0 is None else v0
    for _ in range(n_steps):
        a = policy(x, v, X)[group]
        x, v = BEStep.apply(sim, x, v, a.contiguous())
    reward = x[:, 0].mean() - X[:, 0].mean()
    return reward, x


def train(sim: Simulator, policy: MusclePolicy, X, group, n_steps: int, iters: int, lr: float = 1e-3,
          log=None):
    """Adam on -reward; returns the reward of every iteration (before its update)."""
    opt = torch.optim.Adam(policy.parameters(), lr=lr)
    rewards = []
    for it in range(iters):
        opt.zero_grad()
        reward, _ = episode(sim, policy, X, group, n_steps)
        (-reward).backward()
        opt.step()
        rewards.append(float(reward.detach()))
        if log:
            log(it, rewards[-1])
    return rewards


def _main():
    import synth

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--steps", type=int, default=30, help="backward-Euler steps per episode")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--nx", type=int, default=64)
    ap.add_argument("--ny", type=int, default=32)
    args = ap.parse_args()
    torch.manual_seed(0)
    p = synth.make_config2(n_steps=args.steps, nx=args.nx, ny=args.ny)
    sim = Simulator(p.X, p.T, p.fixed, p.fiber, mu=p.mu, lam=p.lam, k_muscle=p.k_muscle, density=p.density,
                    gravity=p.gravity, k_contact=p.k_contact, contact_power=p.contact_power, dt=p.dt,
                    k_friction=2e3, precision="mixed", adjoint_rtol=1e-8)
    dev = sim.device
    X = torch.from_numpy(p.X).to(dev)
    group = torch.from_numpy(p.extra["group"].astype("int64")).to(dev)
    policy = MusclePolicy(p.n_vert, p.dim, p.extra["n_groups"]).double().to(dev)
    t0 = time.time()
    train(sim, policy, X, group, args.steps, args.iters, lr=args.lr,
          log=lambda it, r: print(f"iter {it:3d}  reward {r:+.6e}  ({time.time() - t0:.1f} s)", flush=True))


if __name__ == "__main__":
    _main()
