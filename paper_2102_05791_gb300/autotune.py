"""Autotuners: the tile shape of the HVP kernel, and the block size of the
batched persistent solver.

For a mesh, tries candidate (elements per tile, threads per block) pairs:
builds a handle for each, runs a short adjoint CG solve at the rest shape
(48 iterations, in whichever way the handle runs CG: one cooperative kernel
when all tiles fit on the GPU, else per-iteration kernels) and keeps the pair
with the smallest time per CG iteration, measured with CUDA events around the
solve.  Results are cached in a JSON file keyed by GPU name, dimension,
element-count bucket (power of two) and precision, so later handles of a
similar mesh reuse the choice without tuning.

    from paper_2102_05791_gb300 import autotune
    te, th = autotune.best_tile_shape(X, T, fixed, fiber, mu=..., lam=..., ...)
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

CANDIDATES = {
    3: [(384, 128), (384, 256), (256, 128), (512, 128), (512, 256), (768, 256)],
    # small tiles give small meshes more CTAs (a 4,096-triangle body has only 8 tiles of 512);
    # at most 16 tiles run the CG solve as one thread-block cluster
    2: [(512, 256), (512, 128), (384, 128), (768, 256), (1024, 256), (256, 256), (256, 128), (128, 128),
        (64, 64)],
}


def cache_path() -> str:
    return os.environ.get("SOFTSIM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "softsim", "autotune.json"))


def _key(dim: int, n_elem: int, precision: str, muscle_model: int = 0) -> str:
    import torch
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    bucket = int(math.log2(max(n_elem, 1)))
    # the spring muscle stages the fiber too (more shared memory per tile)
    return f"{name}|d{dim}|e2^{bucket}|{precision}|per-cg-iteration" + ("|spring" if muscle_model else "")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def measure(X, T, fixed, fiber, tile_elems: int, threads: int, precision: str = "mixed", iters: int = 48,
            **material) -> float:
    """Time per CG iteration (ms) of a short adjoint solve for one tile shape."""
    import torch

    from . import api
    sim = api.Simulator(X, T, fixed, fiber, precision=precision, tile_elems=tile_elems, threads=threads,
                        max_adjoint_cg=iters, adjoint_rtol=1e-30, **material)
    try:
        dev = sim.device
        x = sim.X
        a = torch.zeros(sim.n_elem, dtype=torch.float64, device=dev)
        rng = np.random.default_rng(0)
        b = torch.from_numpy(rng.standard_normal((sim.n_vert, sim.dim))).to(dev)
        sim.adjoint(x, a, b, check=False)  # warm-up: graph capture, module loading
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        _, st = sim.adjoint(x, a, b, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / max(st["cg_iters_total"], 1)
    finally:
        sim.close()


def best_tile_shape(X, T, fixed=None, fiber=None, precision: str = "mixed", candidates=None, use_cache: bool = True,
                    **material):
    """(tile_elems, threads) with the fastest CG iteration for this mesh."""
    X = np.asarray(X)
    T = np.asarray(T)
    dim = X.shape[1]
    key = _key(dim, len(T), precision, int(material.get("muscle_model", 0)))
    cache = _load() if use_cache else {}
    if key in cache:
        return tuple(cache[key]["best"])
    times = {}
    for te, th in (candidates or CANDIDATES[dim]):
        try:
            times[(te, th)] = measure(X, T, fixed, fiber, te, th, precision, **material)
        except Exception:  # a shape this mesh cannot use (e.g. too few threads for a tile)
            times[(te, th)] = float("inf")
    best = min(times, key=times.get)
    if use_cache:
        cache[key] = {"best": list(best), "ms": {f"{k[0]}x{k[1]}": v for k, v in times.items()}}
        _store(cache)
    return best


BATCH_CANDIDATES = (128, 256, 512)


def _batch_key(problems) -> str:
    import torch
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    dim = int(problems[0].X.shape[1])
    n_e = sum(int(p.T.shape[0]) for p in problems)
    return (f"{name}|batch|d{dim}|m2^{int(math.log2(max(len(problems), 1)))}"
            f"|e2^{int(math.log2(max(n_e / max(len(problems), 1), 1)))}")


def measure_batch(problems, threads: int, n_steps: int = 2, **opt) -> float:
    """Milliseconds of one batched rollout + BPTT of n_steps steps (after a warm-up run)."""
    import torch

    from . import api
    b = api.Batch(problems, threads=threads, **opt)
    try:
        dev = b.device
        x0 = torch.from_numpy(np.concatenate([p.X for p in problems])).to(dev)
        v0 = torch.zeros_like(x0)
        rng = np.random.default_rng(0)
        a = torch.from_numpy(rng.uniform(0.2, 0.9, size=(n_steps, b.E))).to(dev)
        xb = torch.from_numpy(rng.standard_normal(tuple(x0.shape))).to(dev)
        b.rollout(x0, v0, a, xb, torch.zeros_like(x0))  # warm-up: graph capture, module loading
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.rollout(x0, v0, a, xb, torch.zeros_like(x0))
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)
    finally:
        b.close()


def best_batch_threads(problems, candidates=None, use_cache: bool = True, **opt) -> int:
    """Threads per mesh CTA with the fastest short batched rollout of these meshes."""
    key = _batch_key(problems)
    cache = _load() if use_cache else {}
    if key in cache:
        return int(cache[key]["best"])
    times = {}
    for th in (candidates or BATCH_CANDIDATES):
        times[th] = measure_batch(problems, th, **opt)
    best = min(times, key=times.get)
    if use_cache:
        cache[key] = {"best": best, "ms": {str(k): v for k, v in times.items()}}
        _store(cache)
    return best
