"""Seeded synthetic meshes and per-element inputs.

The paper's locomotion bodies are not available, so structured grids of the
same kind (triangulated rectangles, tetrahedralised boxes) stand in for them.
Every generator takes an explicit ``numpy.random.Generator`` so that the same
seed gives bit-identical inputs to the oracle and to the GPU path.

Layout conventions (the ones the C ABI uses):

* ``X``      float64 ``[n_vert, d]`` rest positions, row-major; axis 1 (y) is
  vertical, the ground is ``y = 0``.
* ``T``      int32 ``[n_elem, d+1]`` vertex indices, every element positively
  oriented (its rest edge matrix has a positive determinant).
* ``fixed``  uint8 ``[n_vert]``, 1 for Dirichlet (pinned) vertices.
* ``fiber``  float64 ``[n_elem, d]`` unit fiber directions.
* ``a``      float64 ``[n_elem]`` activations.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

BASE_SEED = 20210211

# Material constants of the synthetic workloads (neo-Hookean Lame parameters,
# muscle stiffness, density, gravity, contact stiffness).
MU = 1.0e4
LAMBDA = 4.0e4
K_MUSCLE = 5.0e3
DENSITY = 1.0e3
GRAVITY = 9.8
K_CONTACT = 1.0e6
DT = 1.0 / 30.0


@dataclasses.dataclass
class SynthProblem:
    """One seeded workload: a mesh plus its material and inputs."""

    name: str
    dim: int
    X: np.ndarray          # [nv, d] float64
    T: np.ndarray          # [ne, d+1] int32
    fixed: np.ndarray      # [nv] uint8
    fiber: np.ndarray      # [ne, d] float64
    a: np.ndarray          # [ne] float64
    target: np.ndarray     # [d] float64 loss target for L = 1/2 |mean(x) - target|^2
    mu: float = MU
    lam: float = LAMBDA
    k_muscle: float = K_MUSCLE
    density: float = DENSITY
    gravity: float = GRAVITY
    k_contact: float = 0.0
    contact_power: int = 3
    dt: float = 0.0
    log_mode: int = 0      # 0 = exact log J, 1 = quadratic approximation
    muscle_model: int = 0     # 0 = contractile (k/2) a |Ff|^2, 1 = active spring (k/2)(|Ff|/a - 1)^2
    k_friction: float = 0.0   # ground friction stiffness (dynamics only)
    eps_friction: float = 0.01  # height below which friction acts
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n_vert(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.T.shape[0])


def _jitter_interior(X: np.ndarray, boundary: np.ndarray, h: float,
                     rng: np.random.Generator, amount: float) -> np.ndarray:
    """Move interior vertices by U(-amount, amount) * h per coordinate."""
    if amount <= 0.0:
        return X
    noise = rng.uniform(-amount, amount, size=X.shape) * h
    noise[boundary] = 0.0
    return X + noise


def grid2d(nx: int, ny: int, Lx: float, Ly: float, jitter: float = 0.0,
           rng: np.random.Generator | None = None):
    """Triangulated rectangle [0,Lx]x[0,Ly] with nx*ny cells, 2 triangles each.

    Vertex (i, j) has index i + (nx+1)*j.  Every cell is cut along the diagonal
    from its lower-left to its upper-right corner; both triangles are listed
    counter-clockwise, so they are positively oriented.
    """
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    gx, gy = np.meshgrid(xs, ys, indexing="xy")
    X = np.stack([gx.ravel(), gy.ravel()], axis=1).astype(np.float64)
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    boundary = (ii == 0) | (ii == nx) | (jj == 0) | (jj == ny)
    if rng is not None:
        h = min(Lx / nx, Ly / ny)
        X = _jitter_interior(X, boundary, h, rng, jitter)
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ci = ci.ravel()
    cj = cj.ravel()
    v00 = ci + (nx + 1) * cj
    v10 = v00 + 1
    v01 = v00 + (nx + 1)
    v11 = v01 + 1
    t0 = np.stack([v00, v10, v11], axis=1)
    t1 = np.stack([v00, v11, v01], axis=1)
    T = np.empty((2 * nx * ny, 3), dtype=np.int32)
    T[0::2] = t0
    T[1::2] = t1
    cell_col = np.repeat(ci, 2)
    return X, T, jj.reshape(-1), cell_col


def _lattice_orient(tet):
    """Order four hex-corner offsets so that their signed volume is positive.

    Works on integer corner offsets only (topology of the split, not geometry
    of the jittered mesh).
    """
    a, b, c, d = (np.array(v, dtype=np.int64) for v in tet)
    m = np.stack([b - a, c - a, d - a], axis=1)
    det = (m[0, 0] * (m[1, 1] * m[2, 2] - m[1, 2] * m[2, 1])
           - m[0, 1] * (m[1, 0] * m[2, 2] - m[1, 2] * m[2, 0])
           + m[0, 2] * (m[1, 0] * m[2, 1] - m[1, 1] * m[2, 0]))
    assert det != 0
    if det < 0:
        return (tet[0], tet[2], tet[1], tet[3])
    return tuple(tet)


def _five_tet_templates():
    """5-tet split of a unit hex for even and odd hex parity.

    For even parity the central tet joins the corners whose offset sum is even
    and the four corner tets sit at the odd corners; odd parity mirrors this.
    Neighbouring hexes have opposite parity, so their shared face diagonals
    match and the mesh is conforming.
    """
    corners = list(itertools.product((0, 1), repeat=3))
    out = {}
    for parity in (0, 1):
        centre = [c for c in corners if sum(c) % 2 == parity]
        others = [c for c in corners if sum(c) % 2 != parity]
        tets = [_lattice_orient(centre)]
        for o in others:
            nbrs = [c for c in centre if sum(abs(p - q) for p, q in zip(c, o)) == 1]
            tets.append(_lattice_orient([o] + nbrs))
        out[parity] = tets
    return out


def _six_tet_template():
    """Kuhn (Freudenthal) split: one tet per axis permutation, 000 -> 111."""
    tets = []
    for perm in itertools.permutations(range(3)):
        p0 = (0, 0, 0)
        p1 = list(p0)
        p1[perm[0]] = 1
        p2 = list(p1)
        p2[perm[1]] = 1
        tets.append(_lattice_orient([p0, tuple(p1), tuple(p2), (1, 1, 1)]))
    return tets


def hex_grid3d(nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float,
               split: int = 6, jitter: float = 0.0,
               rng: np.random.Generator | None = None):
    """Tetrahedralised box with nx*ny*nz hexes split into 5 or 6 tets.

    Vertex (i, j, k) has index i + (nx+1)*(j + (ny+1)*k); y (axis 1) is up.
    """
    nvx, nvy, nvz = nx + 1, ny + 1, nz + 1
    xs = np.linspace(0.0, Lx, nvx)
    ys = np.linspace(0.0, Ly, nvy)
    zs = np.linspace(0.0, Lz, nvz)
    kk, jj, ii = np.meshgrid(np.arange(nvz), np.arange(nvy), np.arange(nvx), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    kk = kk.ravel()
    X = np.stack([xs[ii], ys[jj], zs[kk]], axis=1).astype(np.float64)
    boundary = (ii == 0) | (ii == nx) | (jj == 0) | (jj == ny) | (kk == 0) | (kk == nz)
    if rng is not None:
        h = min(Lx / nx, Ly / ny, Lz / nz)
        X = _jitter_interior(X, boundary, h, rng, jitter)

    hk, hj, hi = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    hi = hi.ravel()
    hj = hj.ravel()
    hk = hk.ravel()

    def vid(oi, oj, ok):
        return (hi + oi) + nvx * ((hj + oj) + nvy * (hk + ok))

    if split == 6:
        tmpl = _six_tet_template()
        per_hex = np.stack([np.stack([vid(*c) for c in tet], axis=1) for tet in tmpl], axis=1)
        T = per_hex.reshape(-1, 4)
    elif split == 5:
        tm = _five_tet_templates()
        par = (hi + hj + hk) % 2
        even = np.stack([np.stack([vid(*c) for c in tet], axis=1) for tet in tm[0]], axis=1)
        odd = np.stack([np.stack([vid(*c) for c in tet], axis=1) for tet in tm[1]], axis=1)
        per_hex = np.where(par[:, None, None] == 0, even, odd)
        T = per_hex.reshape(-1, 4)
    else:
        raise ValueError("split must be 5 or 6")
    return X, T.astype(np.int32), jj


def _fibers2d(ne: int, rng: np.random.Generator) -> np.ndarray:
    ang = rng.uniform(0.0, math.pi, size=ne)
    return np.stack([np.cos(ang), np.sin(ang)], axis=1)


def _fibers3d(ne: int, rng: np.random.Generator) -> np.ndarray:
    g = rng.standard_normal((ne, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def _target(X: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    size = X.max(axis=0) - X.min(axis=0)
    return X.mean(axis=0) + rng.uniform(-0.1, 0.1, size=X.shape[1]) * size


def make_small2d(nx: int = 4, ny: int = 2, seed: int = 7, fix_bottom: bool = True,
                 Lx: float = 2.0, Ly: float = 1.0) -> SynthProblem:
    """Tiny jittered 2D problem for brute-force oracle checks."""
    rng = np.random.default_rng(seed)
    X, T, row, _ = grid2d(nx, ny, Lx, Ly, jitter=0.1, rng=rng)
    fixed = (row == 0).astype(np.uint8) if fix_bottom else np.zeros(len(X), np.uint8)
    fiber = _fibers2d(len(T), rng)
    a = rng.uniform(0.0, 1.0, size=len(T))
    return SynthProblem(f"small2d_{nx}x{ny}", 2, X, T, fixed, fiber, a, _target(X, rng))


def make_small3d(nx: int = 2, ny: int = 2, nz: int = 2, split: int = 5, seed: int = 11,
                 fix_bottom: bool = True) -> SynthProblem:
    """Tiny jittered 3D problem for brute-force oracle checks."""
    rng = np.random.default_rng(seed)
    X, T, row = hex_grid3d(nx, ny, nz, 1.0 * nx / ny, 1.0, 1.0 * nz / ny, split=split,
                           jitter=0.1, rng=rng)
    fixed = (row == 0).astype(np.uint8) if fix_bottom else np.zeros(len(X), np.uint8)
    fiber = _fibers3d(len(T), rng)
    a = rng.uniform(0.0, 1.0, size=len(T))
    return SynthProblem(f"small3d_{nx}x{ny}x{nz}_s{split}", 3, X, T, fixed, fiber, a,
                        _target(X, rng))


def make_config1() -> SynthProblem:
    """2D quasistatic: 2.0 x 1.0 rectangle, 16 x 8 cells, 153 vertices, 256 tris."""
    rng = np.random.default_rng(BASE_SEED + 1)
    X, T, row, _ = grid2d(16, 8, 2.0, 1.0, jitter=0.1, rng=rng)
    fixed = (row == 0).astype(np.uint8)
    fiber = _fibers2d(len(T), rng)
    a = rng.uniform(0.0, 1.0, size=len(T))
    return SynthProblem("c1_rect16x8", 2, X, T, fixed, fiber, a, _target(X, rng))


def make_config2(n_steps: int = 200, nx: int = 64, ny: int = 32) -> SynthProblem:
    """2D implicit-Euler dynamics: 64 x 32 grid (2145 vertices, 4096 tris).

    Free body resting on the ground (y = 0), cubic contact penalty, 8 muscle
    groups made of vertical strips of nx/8 cell columns.  ``extra`` holds the
    element -> group map and the per-group sinusoid phases.
    """
    rng = np.random.default_rng(BASE_SEED + 2)
    X, T, _, cell_col = grid2d(nx, ny, 2.0, 1.0, jitter=0.1, rng=rng)
    fixed = np.zeros(len(X), np.uint8)
    fiber = _fibers2d(len(T), rng)
    n_groups = 8
    group = (cell_col * n_groups // nx).astype(np.int32)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=n_groups)
    a_seq = config2_activations(phase, n_steps, DT)
    a0 = a_seq[0][group]
    return SynthProblem("c2_rect64x32_dyn", 2, X, T, fixed, fiber, a0, _target(X, rng),
                        k_contact=K_CONTACT, contact_power=3, dt=DT,
                        extra={"group": group, "phase": phase, "a_groups": a_seq,
                               "n_steps": n_steps, "n_groups": n_groups})


def config2_activations(phase: np.ndarray, n_steps: int, dt: float) -> np.ndarray:
    """a[t, g] = 0.5 + 0.4 sin(2 pi * 1 Hz * t * dt + phase_g)."""
    t = np.arange(n_steps, dtype=np.float64)[:, None]
    return 0.5 + 0.4 * np.sin(2.0 * math.pi * t * dt + phase[None, :])


def make_config3() -> SynthProblem:
    """3D quasistatic: 2 x 1 x 1 box, 32 x 16 x 16 hexes x 5 tets (9537 v, 40960 t)."""
    rng = np.random.default_rng(BASE_SEED + 3)
    X, T, row = hex_grid3d(32, 16, 16, 2.0, 1.0, 1.0, split=5, jitter=0.1, rng=rng)
    fixed = (row == 0).astype(np.uint8)
    fiber = _fibers3d(len(T), rng)
    a = rng.uniform(0.0, 1.0, size=len(T))
    return SynthProblem("c3_box32x16x16_t5", 3, X, T, fixed, fiber, a, _target(X, rng))


# Density of the large 3D body.  With rho = 1e3 its self-weight load
# rho g H / mu is ~2 (H = 2), and the pinned-face edges become so compressed
# (J ~ 0.05 at 128 x 64 x 64) that Newton from rest does not converge; 500
# gives the same load ratio (~1) as the 2 x 1 x 1 box of config 3.
C5_DENSITY = 500.0


def make_config5(scale_div: int = 1) -> SynthProblem:
    """Large 3D quasistatic: 4 x 2 x 2 box, 128 x 64 x 64 hexes x 6 tets.

    ``scale_div = 2`` gives the 1/8-size instance (64 x 32 x 32 hexes) used for
    the full-solve comparison against the oracle.
    """
    rng = np.random.default_rng(BASE_SEED + 5)
    nx, ny, nz = 128 // scale_div, 64 // scale_div, 64 // scale_div
    X, T, row = hex_grid3d(nx, ny, nz, 4.0, 2.0, 2.0, split=6, jitter=0.1, rng=rng)
    fixed = (row == 0).astype(np.uint8)
    fiber = _fibers3d(len(T), rng)
    a = rng.uniform(0.0, 1.0, size=len(T))
    return SynthProblem(f"c5_box{nx}x{ny}x{nz}_t6", 3, X, T, fixed, fiber, a, _target(X, rng),
                        density=C5_DENSITY)


def make_config4(n_meshes: int = 1024, n_steps: int = 60):
    """1024 independent 2D bodies with triangle counts log-uniform in [200, 8000].

    Each body is a 2 x 1 rectangle gridded at its own resolution (aspect 2:1),
    with its own shear modulus mu ~ U(5e3, 2e4), lambda = 4 mu, fibers and a
    seeded sinusoid activation per element.
    """
    rng = np.random.default_rng(BASE_SEED + 4)
    out = []
    for m in range(n_meshes):
        tris = math.exp(rng.uniform(math.log(200.0), math.log(8000.0)))
        cells = tris / 2.0
        ny = max(2, int(round(math.sqrt(cells / 2.0))))
        nx = max(2, int(round(cells / ny)))
        X, T, _, cell_col = grid2d(nx, ny, 2.0, 1.0, jitter=0.1, rng=rng)
        fixed = np.zeros(len(X), np.uint8)
        fiber = _fibers2d(len(T), rng)
        mu = rng.uniform(5.0e3, 2.0e4)
        phase = rng.uniform(0.0, 2.0 * math.pi, size=len(T))
        t = np.arange(n_steps, dtype=np.float64)[:, None]
        a_seq = 0.5 + 0.4 * np.sin(2.0 * math.pi * t * DT + phase[None, :])
        out.append(SynthProblem(f"c4_mesh{m}_{nx}x{ny}", 2, X, T, fixed, fiber, a_seq[0],
                                _target(X, rng), mu=mu, lam=4.0 * mu,
                                k_contact=K_CONTACT, contact_power=3, dt=DT,
                                extra={"a_seq": a_seq, "n_steps": n_steps}))
    return out
