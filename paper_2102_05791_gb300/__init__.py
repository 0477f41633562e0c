"""GB300-native soft-body simulator with implicit differentiation.

Hot path of "Differentiable Implicit Soft-Body Physics" (Rojas, Sifakis,
Kavan, arXiv 2102.05791): neo-Hookean + muscle energy, gradient and
matrix-free Hessian-vector product on triangle / tet meshes, Newton-CG
forward solves, adjoint CG and the parameter VJP, as hand-written CUDA for
sm_103a behind a C ABI (include/softsim.h).  ``build()`` compiles the
library in-tree; ``Simulator`` and the autograd Functions call it.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("Simulator", "QuasistaticSolve", "BEStep", "Rollout", "SimError"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
