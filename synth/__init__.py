"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This package only produces input arrays (meshes, fibers, activations, loss
targets).  It holds none of the simulator's arithmetic: no energy, force,
Hessian or solver code lives here, so the oracle and the CUDA path can both
consume it without sharing any part of the method.
"""
from .meshes import (  # noqa: F401
    BASE_SEED,
    grid2d,
    hex_grid3d,
    SynthProblem,
    make_config1,
    make_config2,
    make_config3,
    make_config4,
    make_config5,
    make_small2d,
    make_small3d,
    config2_activations,
)
