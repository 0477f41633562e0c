"""Helpers shared by the GPU tests: build a Simulator from a seeded problem."""
import numpy as np
import torch


def make_sim(p, precision="fp64", **kw):
    from paper_2102_05791_gb300 import api
    args = dict(mu=p.mu, lam=p.lam, k_muscle=p.k_muscle, density=p.density, gravity=p.gravity,
                k_contact=p.k_contact, contact_power=p.contact_power, log_mode=p.log_mode, dt=p.dt,
                precision=precision)
    args.update(kw)
    return api.Simulator(p.X, p.T, p.fixed, p.fiber, device="cuda:0", **args)


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda:0", dtype=dtype).contiguous()


def host(t):
    return t.detach().cpu().numpy()


def deformed(p, amp, seed):
    """A non-equilibrium state: rest shape plus a smooth field plus noise, pinned vertices at rest."""
    rng = np.random.default_rng(seed)
    X = p.X
    span = X.max(axis=0) - X.min(axis=0)
    s = (X - X.min(axis=0)) / span
    smooth = np.stack([np.sin(2.0 * s[:, (c + 1) % p.dim] + c) for c in range(p.dim)], axis=1) * span.min()
    x = X + amp * smooth + 0.1 * amp * span.min() * rng.standard_normal(X.shape)
    x[p.fixed.astype(bool)] = X[p.fixed.astype(bool)]
    return x
