"""Python face of the FP64 CPU oracle (test infrastructure only).

The arithmetic lives in ``softsim_oracle.c`` (plain element loops, FP64,
single-threaded).  This module compiles it with gcc on first use, loads it
with ctypes and adds the steps that are plain linear algebra on top of it:
dense Hessians on tiny meshes, dense solves, the backward-Euler step and its
backward (Eq. opt-be, Sec. 4), and a fully stored backpropagation through
time over a rollout.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It imports nothing from the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "softsim_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

OK, EINVERTED, ENOTCONVERGED, ELINESEARCH = 0, -3, -4, -5


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("nv", C.c_long), ("ne", C.c_long),
        ("T", C.c_void_p), ("Dminv", C.c_void_p), ("W", C.c_void_p), ("fiber", C.c_void_p),
        ("mass", C.c_void_p), ("fixed", C.c_void_p),
        ("mu", C.c_double), ("lam", C.c_double), ("k_muscle", C.c_double),
        ("gravity", C.c_double), ("k_contact", C.c_double),
        ("contact_power", C.c_int), ("log_mode", C.c_int),
        ("h", C.c_double), ("xhat", C.c_void_p),
        ("muscle_model", C.c_int),
        ("k_friction", C.c_double), ("eps_friction", C.c_double), ("x0", C.c_void_p),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("newton_iters", C.c_int), ("cg_iters_total", C.c_int), ("ls_halvings", C.c_int),
        ("status", C.c_int), ("res0", C.c_double), ("res_final", C.c_double), ("min_J", C.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.c_void_p
        L.or_rest.argtypes = [C.c_int, C.c_long, C.c_long, dp, dp, dp, dp]
        L.or_rest.restype = C.c_int
        L.or_mass.argtypes = [C.c_int, C.c_long, C.c_long, dp, dp, C.c_double, dp]
        L.or_energy.argtypes = [C.POINTER(_Model), dp, dp, dp, dp]
        L.or_energy.restype = C.c_double
        L.or_grad.argtypes = [C.POINTER(_Model), dp, dp, dp, dp]
        L.or_hvp.argtypes = [C.POINTER(_Model), dp, dp, dp, dp]
        L.or_param_vjp.argtypes = [C.POINTER(_Model), dp, dp, dp, dp]
        L.or_material_vjp.argtypes = [C.POINTER(_Model), dp, dp, dp, dp, dp, dp]
        L.or_cg.argtypes = [C.POINTER(_Model), dp, dp, dp, dp, C.c_double, C.c_int, dp]
        L.or_cg.restype = C.c_int
        L.or_newton.argtypes = [C.POINTER(_Model), dp, dp, C.c_double, C.c_int, C.c_int, C.c_int,
                                C.POINTER(Stats)]
        L.or_newton.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclasses.dataclass
class Model:
    """FP64 model of one mesh (rest data computed by the oracle itself)."""

    d: int
    X: np.ndarray
    T: np.ndarray
    Dminv: np.ndarray
    W: np.ndarray
    fiber: np.ndarray
    mass: np.ndarray
    fixed: np.ndarray | None
    mu: float
    lam: float
    k_muscle: float
    gravity: float
    k_contact: float
    contact_power: int
    log_mode: int
    h: float = 0.0
    xhat: np.ndarray | None = None
    k_friction: float = 0.0
    eps_friction: float = 0.01
    x0: np.ndarray | None = None
    muscle_model: int = 0

    @property
    def nv(self):
        return self.X.shape[0]

    @property
    def ne(self):
        return self.T.shape[0]

    def replace(self, **kw) -> "Model":
        return dataclasses.replace(self, **kw)

    def _c(self) -> _Model:
        m = _Model()
        m.d, m.nv, m.ne = self.d, self.nv, self.ne
        m.T, m.Dminv, m.W, m.fiber = _p(self.T), _p(self.Dminv), _p(self.W), _p(self.fiber)
        m.mass = _p(self.mass)
        m.fixed = _p(self.fixed)
        m.mu, m.lam, m.k_muscle = self.mu, self.lam, self.k_muscle
        m.gravity, m.k_contact = self.gravity, self.k_contact
        m.contact_power, m.log_mode = int(self.contact_power), int(self.log_mode)
        m.h = self.h
        m.xhat = _p(self.xhat)
        m.muscle_model = int(self.muscle_model)
        m.k_friction, m.eps_friction = self.k_friction, self.eps_friction
        m.x0 = _p(self.x0)
        return m

    # -- element-level maps -------------------------------------------------
    def energy(self, x, a, with_abs=False):
        x, a = _f64(x), _f64(a)
        S = np.zeros(1)
        mj = np.zeros(1)
        E = lib().or_energy(C.byref(self._c()), _p(x), _p(a), _p(S), _p(mj))
        return (E, S[0]) if with_abs else E

    def min_J(self, x):
        x = _f64(x)
        mj = np.zeros(1)
        lib().or_energy(C.byref(self._c()), _p(x), _p(np.zeros(self.ne)), None, _p(mj))
        return mj[0]

    def grad(self, x, a, with_scale=False):
        x, a = _f64(x), _f64(a)
        g = np.zeros_like(x)
        s = np.zeros_like(x) if with_scale else None
        lib().or_grad(C.byref(self._c()), _p(x), _p(a), _p(g), _p(s))
        return (g, s) if with_scale else g

    def hvp(self, x, a, v):
        x, a, v = _f64(x), _f64(a), _f64(v)
        out = np.zeros_like(x)
        lib().or_hvp(C.byref(self._c()), _p(x), _p(a), _p(v), _p(out))
        return out

    def param_vjp(self, x, lam, a=None):
        """dL/da at x for adjoint lam (a is needed by the spring muscle only)."""
        x, lam = _f64(x), _f64(lam)
        a = np.zeros(self.ne) if a is None else _f64(a)
        out = np.zeros(self.ne)
        lib().or_param_vjp(C.byref(self._c()), _p(x), _p(a), _p(lam), _p(out))
        return out

    def material_vjp(self, x, lam, a):
        """Per-element (dL/dmu, dL/dlambda, dL/dk) at x for adjoint lam."""
        x, lam, a = _f64(x), _f64(lam), _f64(a)
        out = [np.zeros(self.ne) for _ in range(3)]
        lib().or_material_vjp(C.byref(self._c()), _p(x), _p(a), _p(lam), *[_p(o) for o in out])
        return tuple(out)

    # -- solvers ---------------------------------------------------------------
    def cg(self, x, a, b, rtol=1e-10, max_iter=10000):
        x, a, b = _f64(x), _f64(a), _f64(b)
        sol = np.zeros_like(b)
        neg = np.zeros(1, np.int32)
        it = lib().or_cg(C.byref(self._c()), _p(x), _p(a), _p(b), _p(sol), rtol, max_iter, _p(neg))
        return sol, it, bool(neg[0])

    def newton(self, a, x_init=None, rtol=1e-8, max_newton=100, max_cg=None, max_ls=30):
        x = _f64(self.X if x_init is None else x_init).copy()
        a = _f64(a)
        st = Stats()
        if max_cg is None:
            max_cg = int(self.nv * self.d)
        lib().or_newton(C.byref(self._c()), _p(a), _p(x), rtol, max_newton, max_cg, max_ls, C.byref(st))
        return x, st.as_dict()

    def adjoint(self, x_star, a, dLdx, rtol=1e-12, max_iter=None):
        """lambda = H(x*)^-1 dL/dx on free entries (pinned entries stay 0)."""
        b = _f64(dLdx).copy()
        if self.fixed is not None:
            b[self.fixed.astype(bool)] = 0.0
        if max_iter is None:
            max_iter = 4 * int(self.nv * self.d)
        lam, it, neg = self.cg(x_star, a, b, rtol=rtol, max_iter=max_iter)
        return lam, it

    # -- dense (tiny meshes) -----------------------------------------------------
    def dense_hessian(self, x, a):
        """Hessian by columns: H e_j for every unit vector e_j."""
        n = self.nv * self.d
        H = np.zeros((n, n))
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            H[:, j] = self.hvp(x, a, e.reshape(self.nv, self.d)).ravel()
        return H

    def free_mask(self):
        if self.fixed is None:
            return np.ones(self.nv * self.d, bool)
        return np.repeat(self.fixed == 0, self.d)


def make_model(prob, log_mode=None, with_fixed=True, h=None, xhat=None) -> Model:
    """Build the oracle's model of a synth.SynthProblem (rest data by or_rest)."""
    X = _f64(prob.X)
    T = np.ascontiguousarray(prob.T, dtype=np.int32)
    d = prob.dim
    Dminv = np.zeros((len(T), d, d))
    W = np.zeros(len(T))
    rc = lib().or_rest(d, len(X), len(T), _p(X), _p(T), _p(Dminv), _p(W))
    if rc != OK:
        raise ValueError("oracle: element with non-positive rest volume")
    mass = np.zeros(len(X))
    lib().or_mass(d, len(X), len(T), _p(T), _p(W), float(prob.density), _p(mass))
    fixed = np.ascontiguousarray(prob.fixed, dtype=np.uint8) if with_fixed else None
    return Model(d=d, X=X, T=T, Dminv=Dminv, W=W, fiber=_f64(prob.fiber), mass=mass, fixed=fixed,
                 mu=float(prob.mu), lam=float(prob.lam), k_muscle=float(prob.k_muscle),
                 gravity=float(prob.gravity), k_contact=float(prob.k_contact),
                 contact_power=int(prob.contact_power),
                 log_mode=int(prob.log_mode if log_mode is None else log_mode),
                 h=float(prob.dt if h is None else h), xhat=None if xhat is None else _f64(xhat),
                 k_friction=float(getattr(prob, "k_friction", 0.0)),
                 eps_friction=float(getattr(prob, "eps_friction", 0.01)),
                 muscle_model=int(getattr(prob, "muscle_model", 0)))


# ---------------------------------------------------------------------------
# Loss of the synthetic workloads: L = 1/2 |mean(x) - target|^2
# ---------------------------------------------------------------------------

def mean_loss(x, target):
    r = x.mean(axis=0) - target
    return 0.5 * float(r @ r)


def mean_loss_grad(x, target):
    r = x.mean(axis=0) - target
    return np.broadcast_to(r / x.shape[0], x.shape).copy()


def quasistatic_forward_backward(model: Model, a, target, rtol=1e-8, adj_rtol=1e-12):
    """x* = argmin E(., a); lambda = H^-1 dL/dx; dL/da = -lambda^T d2E/dx da."""
    x, st = model.newton(a, rtol=rtol)
    g = mean_loss_grad(x, target)
    lam, it = model.adjoint(x, a, g, rtol=adj_rtol)
    return x, lam, model.param_vjp(x, lam, a), st


# ---------------------------------------------------------------------------
# Backward Euler as an optimisation (Eq. opt-be) and its backward
# ---------------------------------------------------------------------------

def be_step(model: Model, x0, v0, a, rtol=1e-8, max_newton=100):
    """x1 = argmin 1/2 |x - (x0 + h v0)|_M^2 + h^2 E(x, a); v1 = (x1 - x0)/h."""
    h = model.h
    xhat = _f64(x0 + h * v0)
    m = model.replace(xhat=xhat, x0=_f64(x0))
    x1, st = m.newton(a, x_init=x0, rtol=rtol, max_newton=max_newton)
    v1 = (x1 - x0) / h
    return x1, v1, st


def be_step_backward(model: Model, x0, v0, x1, a, xbar1, vbar1, adj_rtol=1e-12, material=False):
    """Adjoint of one backward-Euler step.

    Optimality M (x1 - xhat) + h^2 grad E(x1) = 0 with xhat = x0 + h v0 gives
    (M + h^2 H) dx1 = M dxhat - h^2 (d2E/dx da) da; v1 = (x1 - x0)/h.  With
    lambda = (M + h^2 H)^-1 (xbar1 + vbar1/h):
      xbar0 = M lambda - vbar1/h,  vbar0 = h M lambda,
      abar  = -h^2 lambda^T d2E/dx da.
    With material, also returns the step's (dL/dmu, dL/dlambda, dL/dk) summed
    over the elements (-h^2 lambda^T d2E/dx dtheta).
    """
    h = model.h
    m = model.replace(xhat=_f64(x0 + h * v0), x0=_f64(x0))
    b = xbar1 + vbar1 / h
    lam, it = m.adjoint(x1, a, b, rtol=adj_rtol)
    Ml = model.mass[:, None] * lam
    xbar0 = Ml - vbar1 / h
    if model.k_friction != 0.0:
        # friction depends on x0: h^2 grad_x E_f = fw (x - x0) on horizontal axes,
        # fw = 2 k_f ReLU(eps - y0); xbar0 -= lambda^T d(that)/dx0
        y0 = x0[:, 1]
        active = (model.eps_friction - y0) > 0.0
        fw = 2.0 * model.k_friction * np.where(active, model.eps_friction - y0, 0.0)
        for c in range(x0.shape[1]):
            if c == 1:
                continue
            xbar0[:, c] += fw * lam[:, c]
            xbar0[:, 1] += 2.0 * model.k_friction * active * lam[:, c] * (x1[:, c] - x0[:, c])
    vbar0 = h * Ml
    if model.fixed is not None:
        fx = model.fixed.astype(bool)
        xbar0[fx] = 0.0
        vbar0[fx] = 0.0
    abar = m.param_vjp(x1, lam, a)
    if material:
        return xbar0, vbar0, abar, np.array([v.sum() for v in m.material_vjp(x1, lam, a)])
    return xbar0, vbar0, abar


def rollout(model: Model, x0, v0, a_seq, rtol=1e-8):
    """Fully stored rollout: returns the list of states (x_t, v_t), t = 0..T."""
    xs, vs = [_f64(x0)], [_f64(v0)]
    for t in range(len(a_seq)):
        x1, v1, st = be_step(model, xs[-1], vs[-1], a_seq[t], rtol=rtol)
        if st["status"] != OK:
            raise RuntimeError(f"oracle rollout: step {t} status {st['status']}")
        xs.append(x1)
        vs.append(v1)
    return xs, vs


def rollout_backward(model: Model, xs, vs, a_seq, xbarT, vbarT, adj_rtol=1e-12, material=False):
    """Backpropagation through time over a fully stored rollout.  With
    material, also returns (dL/dmu, dL/dlambda, dL/dk) summed over steps."""
    xbar, vbar = _f64(xbarT), _f64(vbarT)
    abars = [None] * len(a_seq)
    mat = np.zeros(3)
    for t in reversed(range(len(a_seq))):
        out = be_step_backward(model, xs[t], vs[t], xs[t + 1], a_seq[t], xbar, vbar, adj_rtol=adj_rtol,
                               material=material)
        xbar, vbar, abars[t] = out[:3]
        if material:
            mat += out[3]
    if material:
        return xbar, vbar, np.stack(abars), mat
    return xbar, vbar, np.stack(abars)


def horizontal_mean_loss(xT, x0):
    """L = mean_x(x_T) - mean_x(x_0): horizontal centroid displacement."""
    return float(xT[:, 0].mean() - x0[:, 0].mean())


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
