#!/usr/bin/env python3
"""Benchmark of the simulator's hot path on GB300.

One step = one pass of the whole hot path on the large 3D workload: a
Newton-CG quasistatic solve from the rest shape (FP32 HVP inside FP64
Newton control), the loss gradient, the adjoint CG solve and the parameter
VJP.  The workload is a 4 x 2 x 2 box as a 128 x 64 x 64 hex grid, 6 tets per
hex (3,145,728 tets, 545,025 vertices), jittered, neo-Hookean + muscle,
min-y face pinned, gravity on; seeded synthetic inputs.

Printed JSON line (rank 0):
  value      element-HVPs per second over whole steps (n_elem x CG iterations
             of the forward and adjoint solves, divided by the step time);
  e2e        the same through the public API with host buffers, including the
             host<->device copies of every step's inputs and outputs;
  roofline   the HVP tile kernel: algorithmic bytes per launch (72 B per tet +
             36 B per vertex) / its mean duration, against the HBM peak;
  accuracy   the GPU results against the FP64 oracle's own stored solutions
             (tests/golden): the large body at 1/8 size and the config-3 box
             in both precisions, three bodies of the batch, the 200-step
             walker's BPTT gradient, and the mixed CG inner product against
             FP64;
  cpu_baseline  the FP64 oracle on the host cores: element-HVP/s and
             gradient evaluations/s on the large body (one core and all
             cores, one process per core on element slices), and solve wall
             times (single-threaded) on the small workloads.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU (torchrun): every rank solves its own copy of the workload (no
collective on the data path), value = all ranks' element-HVPs / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FALLBACK_HBM_GBS = 6800.0
BYTES_PER_TET = 72.0     # conn 16 + Dm^-1 36 + W 4 + fiber 12 + a 4 (FP32 3D HVP)
BYTES_PER_VERT = 36.0    # read x 12 + read v 12 + write Hv 12
# FP64 HVP arithmetic per tet (3D), counted from the formulas with an FMA as 2 flops:
# edges 18, F 54, dF 45, cof 27, dcof 63, J and dJ 22, log terms ~10, muscle 19,
# stress M 45, G = M B^T + dvg g^T scaled by W 81, p.Ap 18, corner sums 21
FLOPS_PER_TET_FP64 = 420.0
FP64_LANES_PER_SM = 2      # 128 FP32 FMA lanes per SM at 1/64 rate on GB300


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["c5", "c3", "c5_eighth"], default="c5")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 1,024-body measurement")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the comparison with the stored oracle solutions")
    ap.add_argument("--host-cg-loop", action="store_true",
                    help="run every CG solve as host-launched 16-iteration graphs with events around each HVP "
                         "tile launch instead of the device-side WHILE loop (for profilers, which do not see "
                         "kernels inside conditional graph nodes); the printed numbers are then not the bench's")
    ap.add_argument("--cpu-full", action="store_true",
                    help="also time the oracle's 200-step walker BPTT and its 1/8-size large-body solve (minutes)")
    ap.add_argument("--plain-strata", type=int, default=32,
                    help="size strata of the batch sampled for the plain per-mesh FP64 comparison")
    return ap.parse_args()


def workload(name):
    import synth
    if name == "c5":
        return synth.make_config5(), "box 4x2x2, 128x64x64 hex x 6 tets (3,145,728 tets, 545,025 vertices), quasistatic Newton-CG + adjoint + VJP"
    if name == "c5_eighth":
        return synth.make_config5(2), "box 4x2x2, 64x32x32 hex x 6 tets (393,216 tets), quasistatic Newton-CG + adjoint + VJP"
    return synth.make_config3(), "box 2x1x1, 32x16x16 hex x 5 tets (40,960 tets), quasistatic Newton-CG + adjoint + VJP"


def c4_inputs(n_meshes=1024, n_steps=60):
    """1,024 2D bodies (tris log-uniform in [200, 8000], mu ~ U(5e3, 2e4)),
    60 backward-Euler steps, loss = mean horizontal position of each body at
    the end (dL/dx_T = e_x / n_vert per body)."""
    import synth
    probs = synth.make_config4(n_meshes, n_steps)
    x0 = np.concatenate([p.X for p in probs])
    a_seq = np.concatenate([p.extra["a_seq"] for p in probs], axis=1)
    xbT = np.zeros_like(x0)
    off = 0
    for p in probs:
        xbT[off:off + p.n_vert, 0] = 1.0 / p.n_vert
        off += p.n_vert
    return probs, x0, a_seq, xbT


GOLDEN = os.path.join(ROOT, "tests", "golden")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _state_err(x, x_ref, X):
    """max |x - x_ref| over the displacement scale max |x_ref - X|."""
    return float(np.abs(x - x_ref).max() / np.abs(x_ref - X).max())


def run_batched(dev, steps, warmup, n_strata=32):
    """Config 4: one batched launch (forward + BPTT of every body) vs the plain
    per-mesh FP64 path (sim_rollout + sim_rollout_backward per body).  The
    plain path is timed on one body per size stratum (the batch sorted by
    triangle count and cut into n_strata equal groups; the stratum's median
    body stands for its members), so the estimate of the whole batch's plain
    time follows the measured cost-vs-size curve instead of assuming it is
    linear.  A solve = one body-step, forward Newton solve plus adjoint solve.
    Also compares three bodies with the oracle's stored rollouts."""
    import torch
    from paper_2102_05791_gb300 import api
    probs, x0, a_seq, xbT = c4_inputs()
    n_steps = a_seq.shape[0]
    bt = api.Batch(probs, newton_rtol=1e-8, adjoint_rtol=1e-8, threads="auto", device=dev)
    X0 = torch.from_numpy(x0).to(dev)
    V0 = torch.zeros_like(X0)
    A = torch.from_numpy(a_seq).to(dev)
    XB = torch.from_numpy(xbT).to(dev)
    VB = torch.zeros_like(X0)
    states = (torch.empty((n_steps + 1,) + tuple(X0.shape), dtype=torch.float64, device=dev),
              torch.empty((n_steps + 1,) + tuple(X0.shape), dtype=torch.float64, device=dev))
    for _ in range(warmup):
        out = bt.rollout(X0, V0, A, XB, VB, states=states)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        out = bt.rollout(X0, V0, A, XB, VB, states=states)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    mstat = out[5].cpu().numpy()
    solves = len(probs) * n_steps
    res = {"workload": "1,024 2D bodies, tris log-uniform in [200, 8000] (total %d tris), 60 backward-Euler "
                       "steps forward + BPTT" % bt.E,
           "batched_ms_per_rollout": ms, "solves_per_s": solves / (ms / 1e3),
           "threads_per_mesh": bt.threads, "threads_picked_by": "paper_2102_05791_gb300.autotune",
           "bodies_failed": int((mstat[:, 0] != 0).sum()),
           "newton_iters": int(mstat[:, 1].sum()), "cg_iters_fwd": int(mstat[:, 2].sum()),
           "cg_iters_adj": int(mstat[:, 3].sum())}
    acc = None
    gpath = os.path.join(GOLDEN, "c4_bodies_oracle.npz")
    if os.path.exists(gpath):
        g = np.load(gpath)
        sx, ab, vb0 = out[0][-1].cpu().numpy(), out[2].cpu().numpy(), out[4].cpu().numpy()
        vo, eo = bt.vert_offsets, bt.elem_offsets
        per = []
        for k, i in enumerate(g["bodies"]):
            q = probs[i]
            per.append({"body": int(i), "tris": q.n_elem,
                        "state_err": _state_err(sx[vo[i]:vo[i + 1]], g[f"xT_{k}"], q.X),
                        "dLda_rel_l2": _rel(ab[:, eo[i]:eo[i + 1]], g[f"abar_{k}"]),
                        "dLdv0_rel_l2": _rel(vb0[vo[i]:vo[i + 1]], g[f"vbar0_{k}"])})
        acc = {"against": "oracle rollouts + BPTT stored in tests/golden/c4_bodies_oracle.npz (Newton 1e-10, "
                          "adjoints 1e-12)", "bodies": per,
               "max_dLda_rel_l2": max(b["dLda_rel_l2"] for b in per),
               "max_state_err": max(b["state_err"] for b in per)}
    bt.close()
    # plain per-mesh FP64 path, one body per size stratum
    order = np.argsort([p.n_elem for p in probs], kind="stable")
    strata = np.array_split(order, n_strata)
    t_body, tris, t_est = [], [], 0.0
    for members in strata:
        i = members[len(members) // 2]
        p = probs[i]
        sim = api.Simulator(p.X, p.T, p.fixed, p.fiber, mu=p.mu, lam=p.lam, k_muscle=p.k_muscle,
                            density=p.density, gravity=p.gravity, k_contact=p.k_contact,
                            contact_power=p.contact_power, dt=p.dt, precision="fp64", newton_rtol=1e-8,
                            adjoint_rtol=1e-8, device=dev)
        x0i = torch.from_numpy(p.X).to(dev)
        v0i = torch.zeros_like(x0i)
        ai = torch.from_numpy(np.ascontiguousarray(p.extra["a_seq"])).to(dev)
        xbi = torch.zeros_like(x0i)
        xbi[:, 0] = 1.0 / p.n_vert
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xT, vT, ck, _ = sim.rollout(x0i, v0i, ai, ckpt_every=20)
        sim.rollout_backward(ai, ck, 20, xbi, torch.zeros_like(x0i))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sim.close()
        t_body.append(dt)
        tris.append(p.n_elem)
        t_est += dt * len(members)
    # the batched kernel's time split over bodies in proportion to their triangles
    share = np.array(tris, dtype=np.float64) / float(bt.E) * (ms / 1e3)
    ratio = np.array(t_body) / share
    res["plain_fp64_solves_per_s"] = solves / t_est
    res["plain_sample"] = (f"{n_strata} size strata of the batch (sorted by triangle count, equal counts), the "
                           f"median body of each timed through sim_rollout + sim_rollout_backward in FP64 at the "
                           f"same tolerances; batch time = sum over strata of body time x stratum size")
    res["plain_body_seconds"] = {"tris": tris, "seconds": [round(t, 4) for t in t_body]}
    res["speedup_vs_plain_fp64"] = res["solves_per_s"] / res["plain_fp64_solves_per_s"]
    res["speedup_per_body"] = {"min": float(ratio.min()), "median": float(np.median(ratio)),
                               "max": float(ratio.max()),
                               "note": "plain body time / its triangle share of the batched launch"}
    return res, acc


def run_dynamics(dev):
    """Config 2: 64 x 32 grid (4,096 tris), 200 backward-Euler steps with
    checkpoints every 20, forward + BPTT of the horizontal displacement of
    the vertex mean w.r.t. the 8 x 200 group activations (adjoints to 1e-8:
    at 1e-6 the 200-step group gradient was 1.4e-3 off the oracle's)."""
    import torch
    import synth
    from paper_2102_05791_gb300 import api
    p = synth.make_config2()
    group = torch.from_numpy(p.extra["group"].astype(np.int64)).to(dev)
    sim = api.Simulator(p.X, p.T, p.fixed, p.fiber, mu=p.mu, lam=p.lam, k_muscle=p.k_muscle, density=p.density,
                        gravity=p.gravity, k_contact=p.k_contact, contact_power=p.contact_power, dt=p.dt,
                        precision="mixed", adjoint_rtol=1e-8, tile_elems="auto", device=dev)
    a_groups = torch.from_numpy(p.extra["a_groups"]).to(dev)
    x0 = torch.from_numpy(p.X).to(dev)
    a_seq = a_groups[:, group].contiguous()
    # untimed warm-up on the same handle: CUDA-graph capture and module loading,
    # including the group sum (the first index_add_ of a process can spend
    # seconds loading and JIT-compiling PyTorch's kernel for this GPU)
    _, _, ckw, _ = sim.rollout(x0, torch.zeros_like(x0), a_seq[:20].contiguous(), ckpt_every=20)
    _, _, abw, _ = sim.rollout_backward(a_seq[:20].contiguous(), ckw, 20, torch.zeros_like(x0), torch.zeros_like(x0))
    torch.zeros_like(a_groups[:20]).index_add_(1, group, abw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_launch0 = sim.kernel_launches()
    xT, vT, ck, st = sim.rollout(x0, torch.zeros_like(x0), a_seq, ckpt_every=20)
    xbT = torch.zeros_like(x0)
    xbT[:, 0] = 1.0 / p.n_vert
    _, vb0, ab, stb = sim.rollout_backward(a_seq, ck, 20, xbT, torch.zeros_like(x0))
    g = torch.zeros_like(a_groups).index_add_(1, group, ab)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    n_launch = sim.kernel_launches() - n_launch0
    sim.close()
    res = {"workload": "64x32 grid (4,096 tris), 200 backward-Euler steps, checkpoints every 20, forward + BPTT "
                       "(after an untimed 20-step warm-up)", "tile_shape": list(sim.tile_shape),
           "adjoint_rtol": 1e-8, "seconds": dt, "steps_per_s": 200 * 2 / dt,
           "newton_iters": st["newton_iters"] + stb["newton_iters"],
           "cg_iters": st["cg_iters_total"] + stb["cg_iters_total"], "grad_norm": float(g.norm()),
           "gpu_launches": int(n_launch)}
    acc = None
    gpath = os.path.join(GOLDEN, "c2_bptt_oracle.npz")
    if os.path.exists(gpath):
        gg = np.load(gpath)
        acc = {"against": "oracle 200-step rollout + BPTT stored in tests/golden/c2_bptt_oracle.npz (Newton "
                          "1e-10, adjoints 1e-12)",
               "state_err": _state_err(xT.cpu().numpy(), gg["xT"], p.X),
               "dLda_groups_rel_l2": _rel(g.cpu().numpy(), gg["g_groups"]),
               "dLdv0_rel_l2": _rel(vb0.cpu().numpy(), gg["vbar0"])}
    return res, acc


def run_accuracy_quasistatic(dev, name):
    """A quasistatic workload (the large body at 1/8 size, 393,216 tets, or the
    2 x 1 x 1 box of config 3, 40,960 tets): forward solve, adjoint and
    parameter VJP on the GPU in both precisions, against the oracle's stored
    x*, lambda and dL/da (Newton to 1e-10, adjoint to 1e-11)."""
    import torch
    import synth
    from paper_2102_05791_gb300 import api
    gpath = os.path.join(GOLDEN, f"{name}_oracle.npz")
    if not os.path.exists(gpath):
        return None
    g = np.load(gpath)
    if name == "c5_eighth":
        p, desc = synth.make_config5(2), "box 4x2x2, 64x32x32 hex x 6 tets (393,216 tets, 70,785 vertices)"
    else:
        p, desc = synth.make_config3(), "box 2x1x1, 32x16x16 hex x 5 tets (40,960 tets, 9,537 vertices)"
    out = {"against": f"oracle solution stored in tests/golden/{name}_oracle.npz", "workload": desc}
    for prec, kw in (("mixed", {"tile_elems": "auto"}), ("fp64", {"adjoint_rtol": 1e-10})):
        sim = api.Simulator(p.X, p.T, p.fixed, p.fiber, mu=p.mu, lam=p.lam, k_muscle=p.k_muscle,
                            density=p.density, gravity=p.gravity, precision=prec, device=dev, **kw)
        a = torch.from_numpy(p.a).to(dev)
        tgt = torch.from_numpy(p.target).to(dev)
        x, st = sim.solve(a)
        gL = ((x.mean(dim=0) - tgt) / p.n_vert).expand(p.n_vert, p.dim).contiguous()
        lam, sta = sim.adjoint(x, a, gL)
        dLda = sim.param_vjp(x, a, lam)
        xs = x.cpu().numpy()
        out[prec] = {"state_err": _state_err(xs, p.X + g["u_star"], p.X),
                     "lambda_rel_l2": _rel(lam.cpu().numpy(), g["lam"]),
                     "dLda_rel_l2": _rel(dLda.cpu().numpy(), g["dLda"]),
                     "newton_rtol": 1e-8, "adjoint_rtol": kw.get("adjoint_rtol", 1e-6)}
        sim.close()
    return out


def run_dot_accuracy(sim, sim64, x, a, dev):
    """The mixed CG loop's p.Ap (FP32 element quadratic forms, FP32 sums within
    a tile, compensated sums over the tiles) against the FP64 handle's v.(H v)
    at the same state and direction (the FP64 kernels match the oracle to
    1e-12 of the contribution scale)."""
    import torch
    v = torch.from_numpy(np.random.default_rng(17).standard_normal(tuple(x.shape)).astype(np.float32)).to(dev)
    _, q32 = sim.hvp_dot(x, a, v)
    _, q64 = sim64.hvp_dot(x, a, v.double())
    return {"cg_dot_rel_err": abs(q32 - q64) / abs(q64),
            "note": "mixed CG p.Ap vs FP64 v.(H v), large body at the solved state, random direction"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("elem_kernels.cu", "tiling.cpp", "elem_math.cuh", "tile_device.cuh", "layout.h", "tma.cuh",
                  "reduce.cuh", "pdl.cuh", "internal.h")


def kernel_source_hash():
    """Hash of the element-kernel source, the headers it includes and the tile
    builder (which lays out the kernel's inputs), without their // comment
    lines: counters taken on the same code stay valid across comment edits."""
    lines = []
    for f in KERNEL_SOURCES:
        src = os.path.join(ROOT, "paper_2102_05791_gb300", "csrc", f)
        lines += [ln for ln in open(src).read().splitlines() if not ln.strip().startswith("//")]
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def recorded_traffic(workload_name, tile_shape):
    """DRAM bytes per launch of the HVP tile kernel from the committed ncu
    summary, only if it was taken on the current kernel source, workload and
    tile shape (elements per tile, threads); otherwise None."""
    path = os.path.join(ROOT, "profiles", "hvp_tile_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        if (d.get("elem_kernels_sha") == kernel_source_hash() and d.get("workload") == workload_name
                and [d.get("elems_per_tile"), d.get("threads")] == list(tile_shape)):
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def combine_ranks(times, counts, world, device):
    """Whole-job numbers over ranks: the slowest rank's times (max) and the
    summed work counts.  Returns times + counts as floats (identity at N=1)."""
    import torch
    vals = torch.tensor(list(times) + list(counts), dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        t = vals[:len(times)].clone()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        c = vals[len(times):].clone()
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        vals = torch.cat([t, c])
    return [float(v) for v in vals.cpu()]


# ---------------------------------------------------------------- reference arm / CPU baseline
#
# The FP64 oracle on the host cores.  Its checked code stays single-threaded;
# the multi-core figures run one process per core, each on a contiguous slice
# of the large body's elements (the element loop is the whole cost of an HVP
# or gradient evaluation), started together behind a barrier.

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _slice_worker(kind, wl, lo, hi, reps, barrier, queue):
    import oracle
    p, _ = workload(wl)
    m = oracle.make_model(p)
    m = m.replace(T=np.ascontiguousarray(m.T[lo:hi]), Dminv=np.ascontiguousarray(m.Dminv[lo:hi]),
                  W=np.ascontiguousarray(m.W[lo:hi]), fiber=np.ascontiguousarray(m.fiber[lo:hi]))
    a = np.ascontiguousarray(p.a[lo:hi])
    rng = np.random.default_rng(3)
    x = p.X + 1e-3 * rng.standard_normal(p.X.shape)
    v = rng.standard_normal(p.X.shape)
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(reps):
        m.hvp(x, a, v) if kind == "hvp" else m.grad(x, a)
    t1 = time.perf_counter()
    queue.put((t0, t1, hi - lo))


def oracle_rate(kind, n_proc, reps, wl="c5"):
    """Element evaluations per second of the oracle's HVP ("hvp") or gradient
    ("grad") on a workload (default the large body, 3,145,728 tets), n_proc
    processes on element slices: (elements x reps) / (last end - first start)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    ne = workload(wl)[0].n_elem
    cuts = np.linspace(0, ne, n_proc + 1).astype(int)
    barrier, queue = ctx.Barrier(n_proc), ctx.Queue()
    procs = [ctx.Process(target=_slice_worker,
                         args=(kind, wl, int(cuts[i]), int(cuts[i + 1]), reps, barrier, queue))
             for i in range(n_proc)]
    for pr in procs:
        pr.start()
    res = [queue.get() for _ in procs]
    for pr in procs:
        pr.join()
    t0 = min(r[0] for r in res)
    t1 = max(r[1] for r in res)
    return sum(r[2] for r in res) * reps / (t1 - t0), t1 - t0


def _solve_job(name):
    """Single-threaded oracle solves of the small workloads (wall seconds)."""
    import oracle
    import synth
    if name in ("c1", "c3", "c5_eighth"):
        p = {"c1": synth.make_config1, "c3": synth.make_config3,
             "c5_eighth": lambda: synth.make_config5(2)}[name]()
        m = oracle.make_model(p)
        t0 = time.perf_counter()
        oracle.quasistatic_forward_backward(m, p.a, p.target, rtol=1e-8, adj_rtol=1e-6)
        return name, time.perf_counter() - t0, None
    if name == "c2":
        p = synth.make_config2()
        m = oracle.make_model(p)
        a_seq = p.extra["a_groups"][:, p.extra["group"]]
        t0 = time.perf_counter()
        xs, vs = oracle.rollout(m, p.X.copy(), np.zeros_like(p.X), a_seq, rtol=1e-8)
        xb = np.zeros_like(p.X)
        xb[:, 0] = 1.0 / p.n_vert
        oracle.rollout_backward(m, xs, vs, a_seq, xb, np.zeros_like(p.X), adj_rtol=1e-8)
        return name, time.perf_counter() - t0, None
    # c4: the smallest, 10th- and 25th-percentile bodies, sequentially
    probs = synth.make_config4(1024, 60)
    order = np.argsort([q.n_elem for q in probs], kind="stable")
    tris = []
    t0 = time.perf_counter()  # the batch's generation is not part of the solves
    for i in (order[0], order[102], order[256]):
        q = probs[i]
        m = oracle.make_model(q)
        xs, vs = oracle.rollout(m, q.X.copy(), np.zeros_like(q.X), q.extra["a_seq"], rtol=1e-8)
        xb = np.zeros_like(q.X)
        xb[:, 0] = 1.0 / q.n_vert
        oracle.rollout_backward(m, xs, vs, q.extra["a_seq"], xb, np.zeros_like(q.X), adj_rtol=1e-8)
        tris.append(q.n_elem)
    return name, time.perf_counter() - t0, tris


def cpu_baseline(full=False):
    """The oracle as it stands, timed on this host: element-HVP/s and
    gradient evaluations/s on one core and on every core, and single-threaded
    solve wall times (small workloads in parallel processes, one each)."""
    import multiprocessing as mp
    cores = host_cores()
    t_start = time.perf_counter()
    hvp1, _ = oracle_rate("hvp", 1, 3)
    hvpN, _ = oracle_rate("hvp", cores, 3)
    grad1, _ = oracle_rate("grad", 1, 3)
    gradN, _ = oracle_rate("grad", cores, 3)
    jobs = ["c1", "c3", "c4"] + (["c2", "c5_eighth"] if full else [])
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        solved = {n: (t, tr) for n, t, tr in pool.map(_solve_job, jobs)}
    out = {"value": hvpN, "unit": "elem-HVP/s", "cores": cores, "kind": "oracle",
           "sample": (f"FP64 oracle HVP on the large body (3,145,728 tets), 3 evaluations per process; {cores} "
                      f"processes on element slices (one core each) for value, one process for hvp_1core"),
           "hvp_1core": hvp1, "hvp_all_cores": hvpN,
           "grad_per_s_1core": grad1 / 3145728.0, "grad_per_s_all_cores": gradN / 3145728.0,
           "solve_seconds_1core": {
               "c1_quasistatic_fwd_adj": solved["c1"][0],
               "c3_quasistatic_fwd_adj": solved["c3"][0],
               "c4_bodies_60_steps_fwd_bptt": {"tris": solved["c4"][1], "seconds": solved["c4"][0],
                                               "solves_per_s": 3 * 120 / solved["c4"][0]}},
           "tolerances": "Newton 1e-8; adjoint 1e-6 (quasistatic) or 1e-8 (dynamics)",
           "seconds": time.perf_counter() - t_start}
    if full:
        out["solve_seconds_1core"]["c2_200_steps_fwd_bptt"] = solved["c2"][0]
        out["solve_seconds_1core"]["c5_eighth_quasistatic_fwd_adj"] = solved["c5_eighth"][0]
    return out


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands on the host cores, on
    the same workload.  One step = 3 HVP evaluations of the large body on every
    core (element slices, one process per core): the oracle's pure
    element-HVP/s, an upper bound of its whole-step element-HVP/s (a whole
    step also spends time on gradients, energies and vector work)."""
    if rank != 0:
        return
    p, desc = workload(args.workload)
    cores = host_cores()
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt = oracle_rate("hvp", cores, 3, args.workload)
        if i >= args.warmup:
            vals.append((v, dt))
    value = statistics.median(v for v, _ in vals)
    ms = 1000.0 * statistics.median(dt for _, dt in vals)
    sample = (f"pure HVP evaluations of the {args.workload} workload ({p.n_elem} tets), 3 per step, {cores} "
              f"processes on element slices (one core each), FP64 oracle")
    line = {"impl": "reference", "metric": "element-HVP/s (fwd Newton-CG + adjoint, whole step)", "value": value,
            "unit": "elem-HVP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": "elem-HVP/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "elem-HVP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_2102_05791_gb300 import api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p, desc = workload(args.workload)
    sim = api.Simulator(p.X, p.T, p.fixed, p.fiber, mu=p.mu, lam=p.lam, k_muscle=p.k_muscle, density=p.density,
                        gravity=p.gravity, precision=args.precision, tile_elems="auto", device=dev)
    a = torch.from_numpy(p.a).to(dev)
    tgt = torch.from_numpy(p.target).to(dev)
    n = p.n_vert

    def loss_grad(x):
        return ((x.mean(dim=0) - tgt) / n).expand(n, p.dim).contiguous()

    def step(x_init=None, a_in=None):
        x, st = sim.solve(a if a_in is None else a_in, x_init=x_init)
        lam, sta = sim.adjoint(x, a if a_in is None else a_in, loss_grad(x))
        g = sim.param_vjp(x, a if a_in is None else a_in, lam)
        return x, g, st["cg_iters_total"] + sta["cg_iters_total"], st, sta

    def barrier():
        if world > 1:
            dist.barrier()

    if args.host_cg_loop:
        sim.set_kernel_timing(True)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank)
    hvps = 0
    launches0 = sim.kernel_launches()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    last = None
    for _ in range(args.steps):
        x, g, h, st, sta = step()
        hvps += h
        last = (st, sta)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # one more step with CUDA events around every HVP tile launch: the kernel's
    # mean duration inside the solve (the events split the programmatic
    # launch edges into the tile kernel, so this step is kept out of `value`)
    sim.set_kernel_timing(True)
    step()
    torch.cuda.synchronize()
    tile_total_ms, tile_n = sim.kernel_timing()
    sim.set_kernel_timing(args.host_cg_loop)
    launches = sim.kernel_launches() - launches0
    # end-to-end through the public API with host buffers
    X_host = torch.from_numpy(p.X).pin_memory()
    a_host = torch.from_numpy(p.a).pin_memory()
    out_g = torch.empty(p.n_elem, dtype=torch.float64).pin_memory()
    out_x = torch.empty((n, p.dim), dtype=torch.float64).pin_memory()
    e2e_hvps = 0
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        xi = X_host.to(dev, non_blocking=True)
        ai = a_host.to(dev, non_blocking=True)
        x, g, h, _, _ = step(x_init=xi, a_in=ai)
        out_g.copy_(g, non_blocking=True)
        out_x.copy_(x, non_blocking=True)
        e2e_hvps += h
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = f0.elapsed_time(f1)
    # back-to-back launches on the converged state, for comparison only
    b2b_ms, fin_ms = sim.time_hvp(50)
    tile_ms = tile_total_ms / max(tile_n, 1)

    ms, ms_e2e, hvps_all, e2e_all = combine_ranks([ms, ms_e2e], [float(hvps), float(e2e_hvps)], world, dev)
    if rank != 0:
        return
    value = p.n_elem * hvps_all / (ms / 1000.0)
    e2e_value = p.n_elem * e2e_all / (ms_e2e / 1000.0)
    peak, peak_kind = measured_peaks()
    alg_bytes = BYTES_PER_TET * p.n_elem + BYTES_PER_VERT * p.n_vert
    achieved = alg_bytes / (tile_ms / 1000.0) / 1e9
    if args.precision == "fp64":
        # the FP64 HVP is bound by the FP64 pipe (1/64 of the FP32 rate), not by HBM
        props = torch.cuda.get_device_properties(dev)
        sm_mhz = float(clk.get("sm_max_mhz") or 2070.0)
        peak64 = props.multi_processor_count * FP64_LANES_PER_SM * 2.0 * sm_mhz * 1e6 / 1e12
        ach64 = FLOPS_PER_TET_FP64 * p.n_elem / (tile_ms / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s", "frac": ach64 / peak64,
                "traffic": None, "kernel": "k_tile_hvp<double,3>",
                "flops_per_tet": FLOPS_PER_TET_FP64,
                "peak_source": f"derived: {props.multi_processor_count} SMs x {FP64_LANES_PER_SM} FP64 FMA lanes "
                               f"x 2 flops x {sm_mhz:.0f} MHz"}
    else:
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(args.workload, sim.tile_shape), "kernel": "k_tile_hvp<float,3>",
                "peak_source": peak_kind}
    roof.update({"kernel_ms": tile_ms, "kernel_launches_timed": tile_n,
                 "kernel_timing": "CUDA event nodes around every tile launch in one profiled solve after the timed steps",
                 "kernel_ms_back_to_back": b2b_ms})
    line = {
        "metric": "element-HVP/s (fwd Newton-CG + adjoint, whole step)",
        "value": value,
        "unit": "elem-HVP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f32 HVP and CG vectors; CG dot products f32 within a tile or block and compensated f32 across "
                  "them; f64 state, gradient, energies, line search and residual checks")
                 if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": desc, "precision": args.precision,
                   "tile_shape": {"elems_per_tile": sim.tile_shape[0], "threads": sim.tile_shape[1],
                                  "picked_by": "paper_2102_05791_gb300.autotune"},
                   "l2": f"inputs larger than L2: {(BYTES_PER_TET * p.n_elem) / 1e6:.0f} MB element data per HVP"},
        "solves_per_s": world * args.steps / (ms / 1000.0),
        "hvp_per_step": hvps_all / args.steps / world,
        "newton_iters": last[0]["newton_iters"],
        "cg_iters_fwd": last[0]["cg_iters_total"],
        "cg_iters_adj": last[1]["cg_iters_total"],
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": "elem-HVP/s",
                "h2d_bytes_per_step": int(X_host.numel() * 8 + a_host.numel() * 8),
                "d2h_bytes_per_step": int(out_g.numel() * 8 + out_x.numel() * 8),
                # its own solves: the Newton path (and so the HVP count) depends on rounding order
                "hvp_per_step": e2e_all / max(args.steps, 1)},
        "roofline": roof,
        "clocks": clk,
    }
    accuracy = {}
    if not args.no_accuracy and args.workload == "c5":
        # the headline step's CG inner product against the FP64 handle's
        sim64 = api.Simulator(p.X, p.T, p.fixed, p.fiber, mu=p.mu, lam=p.lam, k_muscle=p.k_muscle,
                              density=p.density, gravity=p.gravity, precision="fp64", device=dev)
        xs_last = sim.solve(a)[0]
        accuracy["cg_dot"] = run_dot_accuracy(sim, sim64, xs_last, a, dev)
        sim64.close()
        accuracy["large_body_eighth"] = run_accuracy_quasistatic(dev, "c5_eighth")
        accuracy["box_c3"] = run_accuracy_quasistatic(dev, "c3")
    if not args.no_batched:
        line["batched"], accuracy["batched_bodies"] = run_batched(dev, max(1, min(args.steps, 3)), 1,
                                                                  args.plain_strata)
        line["dynamics"], accuracy["walker_bptt"] = run_dynamics(dev)
    if accuracy:
        line["accuracy"] = accuracy
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_full)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
