"""Run the element HVP of a workload a few times (for timing and profiling).

    python -m paper_2102_05791_gb300.hvp_probe --workload c5 --n 3

Builds the workload's mesh, applies sim_hvp n times at a deformed state with
a random direction, and prints the mean tile/finalize kernel times measured
with CUDA events.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c5", choices=["c5", "c5_eighth", "c3", "c1"])
    ap.add_argument("--n", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tile-elems", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    import numpy as np
    import torch

    import synth
    from paper_2102_05791_gb300 import api
    from paper_2102_05791_gb300.build import build
    build()
    p = {"c5": synth.make_config5, "c5_eighth": lambda: synth.make_config5(2), "c3": synth.make_config3,
         "c1": synth.make_config1}[args.workload]()
    sim = api.Simulator(p.X, p.T, p.fixed, p.fiber, mu=p.mu, lam=p.lam, k_muscle=p.k_muscle, density=p.density,
                        gravity=p.gravity, precision=args.precision, tile_elems=args.tile_elems,
                        threads=args.threads, device="cuda:0")
    rng = np.random.default_rng(0)
    x = torch.from_numpy(p.X + 1e-3 * rng.standard_normal(p.X.shape)).cuda()
    x[torch.from_numpy(p.fixed.astype(bool)).cuda()] = torch.from_numpy(p.X).cuda()[torch.from_numpy(p.fixed.astype(bool)).cuda()]
    a = torch.from_numpy(p.a).cuda()
    v = torch.from_numpy(rng.standard_normal(p.X.shape)).to(device="cuda", dtype=sim.vec_dtype)
    for _ in range(args.n):
        y = sim.hvp(x, a, v)
    torch.cuda.synchronize()
    tile_ms, fin_ms = sim.time_hvp(max(args.n, 1))
    print(f"{args.workload}: {p.n_elem} elements, {p.n_vert} vertices, tiles {sim.tile_stats()}, "
          f"tile {tile_ms * 1e3:.1f} us, finalize {fin_ms * 1e3:.1f} us, |Hv| {float(y.abs().max()):.3e}")


if __name__ == "__main__":
    main()
