"""PyTorch face of libsoftsim: device tensors in, device tensors out.

Every computation runs in the library's CUDA kernels; this module only
checks shapes and dtypes, passes device pointers and the current CUDA stream,
and wraps the solves as ``torch.autograd.Function``s ("physics as a layer",
Sec. 3 of the paper).

Layout: positions and vertex vectors are float64 ``[n_vert, dim]``;
activations and their gradients are float64 ``[n_elem]`` (rollouts:
``[n_steps, n_elem]``).  HVP vectors are float32 for the mixed-precision
handle and float64 for the FP64 handle.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib as L


class SimError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} failed: {L.STATUS_NAMES.get(code, code)} ({msg})")
        self.code = code


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Simulator:
    """One mesh on one GPU (a ``sim_handle``).

    Arguments mirror ``sim_mesh`` / ``sim_material`` / ``sim_options`` in
    include/softsim.h.  Host arrays (numpy or CPU tensors) are copied.
    ``tile_elems="auto"`` (or ``threads="auto"``) picks the tile shape with
    the autotuner (paper_2102_05791_gb300.autotune, cached per GPU).
    ``cg_kernel="auto"`` runs each CG solve as one cooperative kernel when all
    tiles fit on the GPU at once; ``"iteration"`` keeps per-iteration kernels.
    """

    def __init__(self, X, T, fixed=None, fiber=None, *, mu, lam, k_muscle=0.0, density=0.0, gravity=0.0,
                 k_contact=0.0, contact_power=3, log_mode=0, dt=0.0, k_friction=0.0, eps_friction=0.01, muscle_model=0,
                 precision="mixed", newton_rtol=1e-8, newton_forcing=0.5,
                 adjoint_rtol=1e-6, max_newton=100, max_cg=500, max_adjoint_cg=0, max_ls=30, tile_elems=0,
                 threads=0, cg_kernel="auto", device=None):
        self._lib = L.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if tile_elems == "auto" or threads == "auto":
            from . import autotune
            with torch.cuda.device(self.device):
                tile_elems, threads = autotune.best_tile_shape(
                    X, T, fixed, fiber, precision=precision, mu=mu, lam=lam, k_muscle=k_muscle, density=density,
                    gravity=gravity, k_contact=k_contact, contact_power=contact_power, log_mode=log_mode, dt=dt,
                    muscle_model=muscle_model)
        self.tile_shape = (int(tile_elems), int(threads))
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
        T = np.ascontiguousarray(np.asarray(T, dtype=np.int32))
        self.dim = int(X.shape[1])
        self.n_vert = int(X.shape[0])
        self.n_elem = int(T.shape[0])
        fx = None if fixed is None else np.ascontiguousarray(np.asarray(fixed, dtype=np.uint8))
        fb = None if fiber is None else np.ascontiguousarray(np.asarray(fiber, dtype=np.float64))
        mesh = L.SimMesh(self.dim, self.n_vert, self.n_elem, X.ctypes.data, T.ctypes.data,
                         None if fx is None else fx.ctypes.data)
        mat = L.SimMaterial(float(mu), float(lam), float(k_muscle), float(density), float(gravity),
                            float(k_contact), int(contact_power), int(log_mode), float(dt),
                            None if fb is None else fb.ctypes.data, float(k_friction), float(eps_friction),
                            int(muscle_model))
        opt = L.SimOptions()
        self._lib.sim_default_options(C.byref(opt))
        opt.precision = L.SIM_PREC_MIXED if precision == "mixed" else L.SIM_PREC_FP64
        opt.newton_rtol, opt.adjoint_rtol = float(newton_rtol), float(adjoint_rtol)
        opt.newton_forcing = float(newton_forcing)
        opt.max_newton, opt.max_cg, opt.max_adjoint_cg, opt.max_ls = int(max_newton), int(max_cg), int(max_adjoint_cg), int(max_ls)
        opt.tile_elems, opt.threads = int(tile_elems), int(threads)
        opt.cg_kernel = {"auto": L.SIM_CG_AUTO, "iteration": L.SIM_CG_ITERATION}[cg_kernel]
        self.precision = precision
        self.dt = float(dt)
        self.vec_dtype = torch.float32 if precision == "mixed" else torch.float64
        self.X = torch.from_numpy(X).to(self.device)
        self.fixed = None if fx is None else torch.from_numpy(fx).to(self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.sim_create(C.byref(mesh), C.byref(mat), C.byref(opt), C.byref(h))
        if rc != 0:
            raise SimError("sim_create", rc, self._lib.sim_last_error(None).decode())
        self._h = h

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.sim_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def _check(self, fn, rc, allow=()):
        if rc != 0 and rc not in allow:
            raise SimError(fn, rc, self._lib.sim_last_error(self._h).decode())
        return rc

    def _vec(self, t, dtype=torch.float64, name="x"):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
                and tuple(t.shape) == (self.n_vert, self.dim)):
            raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of shape ({self.n_vert}, {self.dim})")
        return t

    def _elem(self, t, name="a"):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and tuple(t.shape) == (self.n_elem,)):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of shape ({self.n_elem},)")
        return t

    def _empty(self, dtype=torch.float64):
        return torch.empty((self.n_vert, self.dim), dtype=dtype, device=self.device)

    # -- element-level maps ------------------------------------------------------
    def energy_grad(self, x, a):
        """(E, grad E) at x (quasistatic energy), FP64."""
        x, a = self._vec(x), self._elem(a)
        E = torch.empty((), dtype=torch.float64, device=self.device)
        g = self._empty()
        self._check("sim_energy_grad", self._lib.sim_energy_grad(self._h, _ptr(x), _ptr(a), _ptr(E), _ptr(g), _stream()))
        return E, g

    def hvp(self, x, a, v):
        """H(x, a) v with pinned rows/columns dropped (vectors in the handle's HVP dtype)."""
        x, a = self._vec(x), self._elem(a)
        v = self._vec(v, self.vec_dtype, "v")
        out = self._empty(self.vec_dtype)
        self._check("sim_hvp", self._lib.sim_hvp(self._h, _ptr(x), _ptr(a), _ptr(v), _ptr(out), _stream()))
        return out

    def hvp_dot(self, x, a, v):
        """(H v, v.(H v)) with the inner product formed as the CG loop forms p.Ap."""
        x, a = self._vec(x), self._elem(a)
        v = self._vec(v, self.vec_dtype, "v")
        out = self._empty(self.vec_dtype)
        q = C.c_double()
        self._check("sim_hvp_dot", self._lib.sim_hvp_dot(self._h, _ptr(x), _ptr(a), _ptr(v), _ptr(out), C.byref(q),
                                                         _stream()))
        return out, q.value

    def material_vjp(self, x_star, a, lam):
        """Per-element (dL/dmu, dL/dlambda, dL/dk) for adjoint lam at x_star."""
        x_star, a, lam = self._vec(x_star), self._elem(a), self._vec(lam, name="lambda")
        outs = [torch.empty(self.n_elem, dtype=torch.float64, device=self.device) for _ in range(3)]
        self._check("sim_material_vjp", self._lib.sim_material_vjp(
            self._h, _ptr(x_star), _ptr(a), _ptr(lam), *[_ptr(o) for o in outs], _stream()))
        return tuple(outs)

    def param_vjp(self, x_star, a, lam):
        x_star, a, lam = self._vec(x_star), self._elem(a), self._vec(lam, name="lambda")
        out = torch.empty(self.n_elem, dtype=torch.float64, device=self.device)
        self._check("sim_param_vjp", self._lib.sim_param_vjp(self._h, _ptr(x_star), _ptr(a), _ptr(lam), _ptr(out),
                                                             _stream()))
        return out

    # -- solves ------------------------------------------------------------------
    def solve(self, a, x_init=None, x0=None, v0=None, check=True):
        """Quasistatic (dt == 0) or backward-Euler (x0, v0 given) Newton-CG solve."""
        a = self._elem(a)
        if x_init is None:
            x_init = self.X if x0 is None else x0
        x_init = self._vec(x_init, name="x_init")
        if x0 is not None:
            x0, v0 = self._vec(x0, name="x0"), self._vec(v0, name="v0")
        out = self._empty()
        st = L.SimStats()
        rc = self._lib.sim_newton_solve(self._h, _ptr(x_init), _ptr(a), _ptr(x0), _ptr(v0), _ptr(out), C.byref(st),
                                        _stream())
        if check:
            self._check("sim_newton_solve", rc)
        return out, st.as_dict()

    def adjoint(self, x_star, a, dLdx, check=True):
        x_star, a, dLdx = self._vec(x_star), self._elem(a), self._vec(dLdx, name="dLdx")
        lam = self._empty()
        st = L.SimStats()
        rc = self._lib.sim_adjoint_solve(self._h, _ptr(x_star), _ptr(a), _ptr(dLdx), _ptr(lam), C.byref(st), _stream())
        if check:
            self._check("sim_adjoint_solve", rc)
        return lam, st.as_dict()

    def step(self, x0, v0, a):
        x0, v0, a = self._vec(x0, name="x0"), self._vec(v0, name="v0"), self._elem(a)
        x1, v1 = self._empty(), self._empty()
        st = L.SimStats()
        self._check("sim_step_forward", self._lib.sim_step_forward(self._h, _ptr(x0), _ptr(v0), _ptr(a), _ptr(x1),
                                                                   _ptr(v1), C.byref(st), _stream()))
        return x1, v1, st.as_dict()

    def step_backward(self, x0, v0, x1, a, xbar1, vbar1):
        xbar0, vbar0 = self._empty(), self._empty()
        abar = torch.empty(self.n_elem, dtype=torch.float64, device=self.device)
        st = L.SimStats()
        self._check("sim_step_backward", self._lib.sim_step_backward(
            self._h, _ptr(self._vec(x0)), _ptr(self._vec(v0)), _ptr(self._vec(x1)), _ptr(self._elem(a)),
            _ptr(self._vec(xbar1)), _ptr(self._vec(vbar1)), _ptr(xbar0), _ptr(vbar0), _ptr(abar), C.byref(st),
            _stream()))
        return xbar0, vbar0, abar, st.as_dict()

    def rollout(self, x0, v0, a_seq, ckpt_every=20):
        x0, v0 = self._vec(x0, name="x0"), self._vec(v0, name="v0")
        a_seq = a_seq.contiguous()
        n_steps = int(a_seq.shape[0])
        assert a_seq.dtype == torch.float64 and a_seq.shape[1:] == (self.n_elem,)
        n_ckpt = max(1, math.ceil(n_steps / ckpt_every))
        ck_x = torch.empty((n_ckpt, self.n_vert, self.dim), dtype=torch.float64, device=self.device)
        ck_v = torch.empty_like(ck_x)
        xT, vT = self._empty(), self._empty()
        st = L.SimStats()
        self._check("sim_rollout", self._lib.sim_rollout(self._h, n_steps, _ptr(x0), _ptr(v0), _ptr(a_seq), ckpt_every,
                                                         _ptr(ck_x), _ptr(ck_v), _ptr(xT), _ptr(vT), C.byref(st),
                                                         _stream()))
        return xT, vT, (ck_x, ck_v), st.as_dict()

    def rollout_backward(self, a_seq, ckpt, ckpt_every, xbarT, vbarT):
        a_seq = a_seq.contiguous()
        n_steps = int(a_seq.shape[0])
        ck_x, ck_v = ckpt
        seg_x = torch.empty((ckpt_every + 1, self.n_vert, self.dim), dtype=torch.float64, device=self.device)
        seg_v = torch.empty_like(seg_x)
        xbar0, vbar0 = self._empty(), self._empty()
        abar = torch.empty_like(a_seq)
        st = L.SimStats()
        self._check("sim_rollout_backward", self._lib.sim_rollout_backward(
            self._h, n_steps, _ptr(a_seq), ckpt_every, _ptr(ck_x), _ptr(ck_v), _ptr(self._vec(xbarT.contiguous())),
            _ptr(self._vec(vbarT.contiguous())), _ptr(xbar0), _ptr(vbar0), _ptr(abar), _ptr(seg_x), _ptr(seg_v),
            C.byref(st), _stream()))
        return xbar0, vbar0, abar, st.as_dict()

    # -- diagnostics -------------------------------------------------------------
    def time_hvp(self, n=20):
        ms = (C.c_float * 2)()
        self._check("sim_time_hvp", self._lib.sim_time_hvp(self._h, int(n), ms, _stream()))
        return float(ms[0]), float(ms[1])

    def set_kernel_timing(self, on=True):
        self._check("sim_set_kernel_timing", self._lib.sim_set_kernel_timing(self._h, int(bool(on))))

    def kernel_timing(self):
        """(summed ms, launches) of HVP tile kernels timed inside solves."""
        ms, n = C.c_double(), C.c_int64()
        self._lib.sim_kernel_timing(self._h, C.byref(ms), C.byref(n))
        return float(ms.value), int(n.value)

    def set_wait_limit(self, polls):
        """Poll limit of the HVP tile kernel's first bulk-copy wait (testing aid;
        negative restores the default)."""
        self._check("sim_set_wait_limit", self._lib.sim_set_wait_limit(self._h, int(polls)))

    def kernel_launches(self):
        n = C.c_int64()
        self._lib.sim_counters(self._h, C.byref(n))
        return int(n.value)

    def tile_stats(self):
        n = C.c_int()
        e, v, hf = C.c_double(), C.c_double(), C.c_double()
        self._lib.sim_tile_stats(self._h, C.byref(n), C.byref(e), C.byref(v), C.byref(hf))
        return {"n_tiles": n.value, "elems_per_tile": e.value, "verts_per_tile": v.value, "halo_fraction": hf.value}


class Batch:
    """Many meshes rolled out and differentiated in one persistent launch (sim_batch_*).

    ``problems`` are dicts or objects with X, T, fixed, fiber, mu, lam and the
    shared scalars (k_muscle, density, gravity, k_contact, contact_power,
    log_mode, dt).  Concatenated layouts follow include/softsim.h.
    """

    def __init__(self, problems, newton_rtol=1e-8, adjoint_rtol=1e-6, max_newton=100, max_cg=500,
                 max_adjoint_cg=2000, max_ls=30, threads=0, device=None):
        self._lib = L.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if threads == "auto":
            from . import autotune
            with torch.cuda.device(self.device):
                threads = autotune.best_batch_threads(problems, newton_rtol=newton_rtol, adjoint_rtol=adjoint_rtol,
                                                      max_newton=max_newton, max_cg=max_cg,
                                                      max_adjoint_cg=max_adjoint_cg, max_ls=max_ls)
        self.threads = int(threads) if threads else 256
        self._keep = []
        n = len(problems)
        meshes = (L.SimMesh * n)()
        mats = (L.SimMaterial * n)()
        for i, p in enumerate(problems):
            X = np.ascontiguousarray(p.X, dtype=np.float64)
            T = np.ascontiguousarray(p.T, dtype=np.int32)
            fx = np.ascontiguousarray(p.fixed, dtype=np.uint8)
            fb = np.ascontiguousarray(p.fiber, dtype=np.float64)
            self._keep += [X, T, fx, fb]
            meshes[i] = L.SimMesh(X.shape[1], X.shape[0], T.shape[0], X.ctypes.data, T.ctypes.data, fx.ctypes.data)
            mats[i] = L.SimMaterial(p.mu, p.lam, p.k_muscle, p.density, p.gravity, p.k_contact, p.contact_power,
                                    p.log_mode, p.dt, fb.ctypes.data, float(getattr(p, "k_friction", 0.0)),
                                    float(getattr(p, "eps_friction", 0.01)), int(getattr(p, "muscle_model", 0)))
        opt = L.SimOptions()
        self._lib.sim_default_options(C.byref(opt))
        opt.newton_rtol, opt.adjoint_rtol = float(newton_rtol), float(adjoint_rtol)
        opt.max_newton, opt.max_cg, opt.max_adjoint_cg, opt.max_ls = int(max_newton), int(max_cg), int(max_adjoint_cg), int(max_ls)
        opt.threads = self.threads
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.sim_batch_create(n, meshes, mats, C.byref(opt), C.byref(h))
        if rc != 0:
            raise SimError("sim_batch_create", rc, self._lib.sim_batch_last_error(None).decode())
        self._h = h
        self._keep = []
        nm, V, E = C.c_int(), C.c_int64(), C.c_int64()
        self._lib.sim_batch_sizes(h, C.byref(nm), C.byref(V), C.byref(E))
        self.n_meshes, self.V, self.E = nm.value, V.value, E.value
        self.dim = problems[0].X.shape[1]
        self.vert_offsets = np.concatenate([[0], np.cumsum([p.X.shape[0] for p in problems])])
        self.elem_offsets = np.concatenate([[0], np.cumsum([p.T.shape[0] for p in problems])])

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sim_batch_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def rollout(self, x0, v0, a_seq, xbarT, vbarT, states=None, material_grad=False):
        """Forward rollout + BPTT of every mesh.  Returns (states_x, states_v,
        abar_seq, xbar0, vbar0, mesh_stats) as device tensors, plus, with
        material_grad, the [n_meshes, 3] per-mesh (dL/dmu, dL/dlambda, dL/dk)."""
        n_steps = int(a_seq.shape[0])
        if states is None:
            sx = torch.empty((n_steps + 1, self.V, self.dim), dtype=torch.float64, device=self.device)
            sv = torch.empty_like(sx)
        else:
            sx, sv = states
        sx[0].copy_(x0)
        sv[0].copy_(v0)
        a_seq = a_seq.contiguous()
        abar = torch.empty_like(a_seq)
        xb0 = torch.empty((self.V, self.dim), dtype=torch.float64, device=self.device)
        vb0 = torch.empty_like(xb0)
        ms = torch.zeros((self.n_meshes, 4), dtype=torch.int32, device=self.device)
        mg = torch.empty((self.n_meshes, 3), dtype=torch.float64, device=self.device) if material_grad else None
        rc = self._lib.sim_batch_rollout(self._h, n_steps, _ptr(sx), _ptr(sv), _ptr(a_seq),
                                         _ptr(xbarT.contiguous()), _ptr(vbarT.contiguous()), _ptr(abar), _ptr(xb0),
                                         _ptr(vb0), _ptr(ms), None if mg is None else _ptr(mg), _stream())
        if rc != 0:
            raise SimError("sim_batch_rollout", rc, self._lib.sim_batch_last_error(self._h).decode())
        return (sx, sv, abar, xb0, vb0, ms, mg) if material_grad else (sx, sv, abar, xb0, vb0, ms)


# ---------------------------------------------------------------- autograd

class QuasistaticSolve(torch.autograd.Function):
    """x* = argmin_x E(x, a); backward dL/da = -(H^-1 dL/dx)^T d2E/dx da (Eq. dLda-re-ordered)."""

    @staticmethod
    def forward(ctx, sim: Simulator, a):
        x, st = sim.solve(a.detach().contiguous())
        ctx.sim = sim
        ctx.save_for_backward(x, a)
        return x

    @staticmethod
    def backward(ctx, gx):
        x, a = ctx.saved_tensors
        lam, _ = ctx.sim.adjoint(x, a.detach().contiguous(), gx.contiguous())
        return None, ctx.sim.param_vjp(x, a.detach().contiguous(), lam)


class BEStep(torch.autograd.Function):
    """(x1, v1) = backward-Euler step (Eq. opt-be) with its implicit-differentiation backward."""

    @staticmethod
    def forward(ctx, sim: Simulator, x0, v0, a):
        x0c, v0c, ac = x0.detach().contiguous(), v0.detach().contiguous(), a.detach().contiguous()
        x1, v1, _ = sim.step(x0c, v0c, ac)
        ctx.sim = sim
        ctx.save_for_backward(x0c, v0c, x1, ac)
        return x1, v1

    @staticmethod
    def backward(ctx, gx1, gv1):
        x0, v0, x1, a = ctx.saved_tensors
        gx1 = torch.zeros_like(x1) if gx1 is None else gx1.contiguous()
        gv1 = torch.zeros_like(x1) if gv1 is None else gv1.contiguous()
        xb0, vb0, ab, _ = ctx.sim.step_backward(x0, v0, x1, a, gx1, gv1)
        return None, xb0, vb0, ab


class Rollout(torch.autograd.Function):
    """T backward-Euler steps with checkpoints every `ckpt_every` steps; the
    backward recomputes each segment from its checkpoint (memory O(T/k + k))."""

    @staticmethod
    def forward(ctx, sim: Simulator, x0, v0, a_seq, ckpt_every=20):
        xT, vT, ckpt, _ = sim.rollout(x0.detach().contiguous(), v0.detach().contiguous(),
                                      a_seq.detach().contiguous(), ckpt_every)
        ctx.sim, ctx.k = sim, ckpt_every
        ctx.save_for_backward(a_seq.detach().contiguous(), *ckpt)
        return xT, vT

    @staticmethod
    def backward(ctx, gxT, gvT):
        a_seq, ck_x, ck_v = ctx.saved_tensors
        gxT = torch.zeros_like(ck_x[0]) if gxT is None else gxT
        gvT = torch.zeros_like(ck_x[0]) if gvT is None else gvT
        xb0, vb0, ab, _ = ctx.sim.rollout_backward(a_seq, (ck_x, ck_v), ctx.k, gxT, gvT)
        return None, xb0, vb0, ab, None
