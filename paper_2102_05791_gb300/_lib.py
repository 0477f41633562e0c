"""ctypes declarations of libsoftsim (the C ABI in include/softsim.h).

Argument marshalling only.  Loading fails loudly when the library has not
been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsoftsim.so")

SIM_OK, SIM_EINVAL, SIM_ECUDA, SIM_EINVERTED, SIM_ENOTCONVERGED, SIM_ELINESEARCH, SIM_ENAN, SIM_ENOMEM = (
    0, -1, -2, -3, -4, -5, -6, -7)
SIM_PREC_FP64, SIM_PREC_MIXED = 0, 1
SIM_LOG_EXACT, SIM_LOG_QUAD = 0, 1
SIM_MUSCLE_CONTRACTILE, SIM_MUSCLE_SPRING = 0, 1
SIM_CG_AUTO, SIM_CG_ITERATION = 0, 1

STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ECUDA", -3: "EINVERTED", -4: "ENOTCONVERGED",
                -5: "ELINESEARCH", -6: "ENAN", -7: "ENOMEM"}

EXPORTED = [
    "sim_default_options", "sim_create", "sim_destroy", "sim_last_error", "sim_sizes",
    "sim_energy_grad", "sim_hvp", "sim_hvp_dot", "sim_newton_solve", "sim_adjoint_solve", "sim_param_vjp", "sim_material_vjp",
    "sim_step_forward", "sim_step_backward", "sim_rollout", "sim_rollout_backward",
    "sim_time_hvp", "sim_tile_stats", "sim_counters", "sim_energy_noalloc", "sim_noalloc_last_error",
    "sim_set_kernel_timing", "sim_kernel_timing", "sim_set_wait_limit",
    "sim_batch_create", "sim_batch_destroy", "sim_batch_last_error", "sim_batch_sizes", "sim_batch_rollout",
]


class SimMesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_vert", C.c_int64), ("n_elem", C.c_int64),
                ("rest_pos", C.c_void_p), ("elems", C.c_void_p), ("fixed", C.c_void_p)]


class SimMaterial(C.Structure):
    _fields_ = [("mu", C.c_double), ("lambda_", C.c_double), ("k_muscle", C.c_double),
                ("density", C.c_double), ("gravity", C.c_double), ("k_contact", C.c_double),
                ("contact_power", C.c_int), ("log_mode", C.c_int), ("dt", C.c_double),
                ("fiber", C.c_void_p), ("k_friction", C.c_double), ("eps_friction", C.c_double),
                ("muscle_model", C.c_int)]


class SimOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("newton_rtol", C.c_double), ("newton_forcing", C.c_double),
                ("adjoint_rtol", C.c_double),
                ("max_newton", C.c_int), ("max_cg", C.c_int), ("max_adjoint_cg", C.c_int),
                ("max_ls", C.c_int), ("tile_elems", C.c_int), ("threads", C.c_int), ("cg_kernel", C.c_int)]


class SimStats(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("cg_iters_total", C.c_int), ("ls_halvings", C.c_int),
                ("status", C.c_int), ("res0", C.c_double), ("res_final", C.c_double),
                ("min_J", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(path: str | None = None):
    """Load libsoftsim.so (built in-tree by paper_2102_05791_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libsoftsim.so not found at {p}: run paper_2102_05791_gb300.build.build() first")
    L = C.CDLL(p)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    H = C.c_void_p
    L.sim_default_options.argtypes = [C.POINTER(SimOptions)]
    L.sim_create.argtypes = [C.POINTER(SimMesh), C.POINTER(SimMaterial), C.POINTER(SimOptions), C.POINTER(H)]
    L.sim_destroy.argtypes = [H]
    L.sim_last_error.argtypes = [H]
    L.sim_last_error.restype = C.c_char_p
    L.sim_sizes.argtypes = [H, C.POINTER(i), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.sim_energy_grad.argtypes = [H, vp, vp, vp, vp, vp]
    L.sim_hvp.argtypes = [H, vp, vp, vp, vp, vp]
    L.sim_hvp_dot.argtypes = [H, vp, vp, vp, vp, C.POINTER(d), vp]
    L.sim_newton_solve.argtypes = [H, vp, vp, vp, vp, vp, C.POINTER(SimStats), vp]
    L.sim_adjoint_solve.argtypes = [H, vp, vp, vp, vp, C.POINTER(SimStats), vp]
    L.sim_param_vjp.argtypes = [H, vp, vp, vp, vp, vp]
    L.sim_material_vjp.argtypes = [H, vp, vp, vp, vp, vp, vp, vp]
    L.sim_step_forward.argtypes = [H, vp, vp, vp, vp, vp, C.POINTER(SimStats), vp]
    L.sim_step_backward.argtypes = [H, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(SimStats), vp]
    L.sim_rollout.argtypes = [H, i, vp, vp, vp, i, vp, vp, vp, vp, C.POINTER(SimStats), vp]
    L.sim_rollout_backward.argtypes = [H, i, vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(SimStats), vp]
    L.sim_time_hvp.argtypes = [H, i, C.POINTER(C.c_float), vp]
    L.sim_counters.argtypes = [H, C.POINTER(C.c_int64)]
    L.sim_set_kernel_timing.argtypes = [H, i]
    L.sim_kernel_timing.argtypes = [H, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.sim_set_wait_limit.argtypes = [H, i]
    L.sim_energy_noalloc.argtypes = [i, C.c_int64, C.c_int64, vp, vp, vp, vp, vp, C.POINTER(SimMaterial), vp, vp]
    L.sim_noalloc_last_error.argtypes = []
    L.sim_noalloc_last_error.restype = C.c_char_p
    L.sim_tile_stats.argtypes = [H, C.POINTER(i), C.POINTER(d), C.POINTER(d), C.POINTER(d)]
    L.sim_batch_create.argtypes = [i, C.POINTER(SimMesh), C.POINTER(SimMaterial), C.POINTER(SimOptions), C.POINTER(H)]
    L.sim_batch_destroy.argtypes = [H]
    L.sim_batch_last_error.argtypes = [H]
    L.sim_batch_last_error.restype = C.c_char_p
    L.sim_batch_sizes.argtypes = [H, C.POINTER(i), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.sim_batch_rollout.argtypes = [H, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    for name in EXPORTED:
        if name not in ("sim_last_error", "sim_noalloc_last_error", "sim_batch_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L
