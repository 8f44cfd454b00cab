"""Seeded synthetic inputs for the mass-spring cloth workloads.

This module produces problem *inputs* only: grid placement, masses, spring
constants, pins, initial positions, wind parameters and static surface meshes.
It holds none of the method's arithmetic (no spring forces, no integration, no
collision); the CUDA library and the CPU oracle each implement the method on
their own and both read the arrays produced here.

Surface models.  The paper collides the cloth with three baked triangle models
(a 0.9K-triangle sphere, the 50.6K-triangle Armadillo and the 100K-triangle
Dragon, Section 4.2).  Those meshes are not available, so seeded icospheres
stand in for them: level L of midpoint subdivision has 20*4^L triangles
(L2 = 320, L4 = 5,120, L5 = 20,480, L6 = 81,920), optionally displaced
radially by Perlin's improved gradient noise (Perlin 2002, "Improving Noise").

Cloth.  A regular nx-by-ny grid of nodes (node id = row*nx + col) placed at
``origin + col*du + row*dv``, the grid cloth of the paper's hanging-cloth and
collision experiments (Section 4.1, 4.2) at the resolutions the workloads name.
"""
from __future__ import annotations

import dataclasses
import functools
import math
from typing import List, Optional, Tuple

import numpy as np

# ---------------------------------------------------------------------------
# Meshes
# ---------------------------------------------------------------------------


def _icosahedron() -> Tuple[np.ndarray, np.ndarray]:
    """Unit icosahedron: 12 vertices, 20 outward-oriented faces (sorted)."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-g, g):
            v.append((a, b, 0.0))
            v.append((0.0, a, b))
            v.append((b, 0.0, a))
    v = np.array(v, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    n = len(v)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    edge = np.min(d[d > 1e-9])
    adj = np.abs(d - edge) < 1e-6
    faces = []
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    a, b, c = v[i], v[j], v[k]
                    if np.dot(np.cross(b - a, c - a), a + b + c) < 0:
                        faces.append((i, k, j))
                    else:
                        faces.append((i, j, k))
    f = np.array(faces, dtype=np.int64)
    assert f.shape == (20, 3)
    return v, f


def icosphere(level: int) -> Tuple[np.ndarray, np.ndarray]:
    """Unit icosphere by midpoint subdivision + projection, in FP64.

    Returns (verts float64 (10*4^L+2, 3), tris int32 (20*4^L, 3)); faces are
    oriented outward and each face of level L-1 becomes 4 consecutive faces.
    (Cached per level; callers get copies.)
    """
    v, f = _icosphere_cached(int(level))
    return v.copy(), f.copy()


@functools.lru_cache(maxsize=None)
def _icosphere_cached(level: int) -> Tuple[np.ndarray, np.ndarray]:
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    for _ in range(level):
        cache = {}

        def mid(i: int, j: int) -> int:
            key = (i, j) if i < j else (j, i)
            if key in cache:
                return cache[key]
            p = (np.array(verts[i]) + np.array(verts[j])) * 0.5
            p /= np.linalg.norm(p)
            verts.append(tuple(p))
            cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = np.array(nf, dtype=np.int64)
    return np.array(verts, dtype=np.float64), f.astype(np.int32)


def _perlin_fade(t):
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def _perlin_grad(h, x, y, z):
    h = h & 15
    u = np.where(h < 8, x, y)
    v = np.where(h < 4, y, np.where((h == 12) | (h == 14), x, z))
    return np.where((h & 1) == 0, u, -u) + np.where((h & 2) == 0, v, -v)


def perlin_noise3(p: np.ndarray, seed: int) -> np.ndarray:
    """Perlin's improved gradient noise at points p (M,3), values in ~[-1,1].

    The 256-entry permutation is ``numpy.random.default_rng(seed)
    .permutation(256)`` (doubled), replacing Perlin's fixed table; fade curve
    6t^5-15t^4+10t^3 and the 12 edge gradients follow the published method.
    """
    perm = np.random.default_rng(seed).permutation(256).astype(np.int64)
    P = np.concatenate([perm, perm])
    fl = np.floor(p)
    X = fl[:, 0].astype(np.int64) & 255
    Y = fl[:, 1].astype(np.int64) & 255
    Z = fl[:, 2].astype(np.int64) & 255
    x = p[:, 0] - fl[:, 0]
    y = p[:, 1] - fl[:, 1]
    z = p[:, 2] - fl[:, 2]
    u, v, w = _perlin_fade(x), _perlin_fade(y), _perlin_fade(z)
    A = P[X] + Y
    AA = P[A] + Z
    AB = P[A + 1] + Z
    B = P[X + 1] + Y
    BA = P[B] + Z
    BB = P[B + 1] + Z

    def lerp(t, a, b):
        return a + t * (b - a)

    return lerp(
        w,
        lerp(v,
             lerp(u, _perlin_grad(P[AA], x, y, z), _perlin_grad(P[BA], x - 1, y, z)),
             lerp(u, _perlin_grad(P[AB], x, y - 1, z), _perlin_grad(P[BB], x - 1, y - 1, z))),
        lerp(v,
             lerp(u, _perlin_grad(P[AA + 1], x, y, z - 1), _perlin_grad(P[BA + 1], x - 1, y, z - 1)),
             lerp(u, _perlin_grad(P[AB + 1], x, y - 1, z - 1), _perlin_grad(P[BB + 1], x - 1, y - 1, z - 1))),
    )


def sphere_mesh(level: int, radius: float, center=(0.0, 0.0, 0.0),
                noise_amp: float = 0.0, noise_seed: int = 0,
                noise_freq: float = 3.0) -> Tuple[np.ndarray, np.ndarray]:
    """Icosphere of ``radius`` (optionally displaced) at ``center``.

    Displacement: r(s) = radius + noise_amp * n(noise_freq * s) for the unit
    direction s.  Built in FP64 and returned as float32 verts / int32 tris,
    the arrays both the GPU library and the oracle receive.
    """
    v, f = icosphere(level)
    r = np.full(len(v), float(radius))
    if noise_amp != 0.0:
        r = r + noise_amp * perlin_noise3(noise_freq * v, noise_seed)
    out = v * r[:, None] + np.asarray(center, dtype=np.float64)[None, :]
    return out.astype(np.float32), f.astype(np.int32)


# ---------------------------------------------------------------------------
# Cloth scenes
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Wind:
    """w(X0, t) = amp * dir * sin(2*pi*freq*t + kappa*(udir . X0) + phase)."""
    amp: float = 0.0
    dir: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    udir: Tuple[float, float, float] = (1.0, 0.0, 0.0)
    freq: float = 0.0
    kappa: float = 0.0
    phase: float = 0.0


@dataclasses.dataclass
class Scene:
    """One cloth problem: everything the paper's problem statement needs.

    Arrays are float32 / int32 / uint8 exactly as both implementations read
    them; scalars are Python floats that each side rounds to its own precision.
    """
    name: str
    nx: int
    ny: int
    origin: Tuple[float, float, float]
    du: Tuple[float, float, float]
    dv: Tuple[float, float, float]
    total_mass: float
    ks: Tuple[float, float, float]          # structural, shear, bend (N/m)
    kd: Tuple[float, float, float]          # (N s/m)
    gravity: Tuple[float, float, float]
    dt: float
    substeps: int
    steps: int
    init_pos: np.ndarray                    # float32 (N,3)
    init_vel: np.ndarray                    # float32 (N,3)
    pinned: np.ndarray                      # uint8 (N,)
    mesh_verts: Optional[np.ndarray] = None  # float32 (V,3)
    mesh_tris: Optional[np.ndarray] = None   # int32 (T,3)
    ks_spring: Optional[np.ndarray] = None   # float32 (S,), canonical order
    kd_spring: Optional[np.ndarray] = None
    contact_offset: float = 1e-4
    mt_eps: float = 1e-7       # parallel test |a| < eps of the extended MT test
    mt_t_min: float = 0.0      # hit distance bound t_min < t < |d|
    restitution: float = -0.5
    wind: Wind = dataclasses.field(default_factory=Wind)
    pin_velocity: Tuple[float, float, float] = (0.0, 0.0, 0.0)  # pinned nodes move at this velocity (m/s)

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def dt_s(self) -> float:
        return self.dt / self.substeps

    @property
    def ntris(self) -> int:
        return 0 if self.mesh_tris is None else int(len(self.mesh_tris))


def spring_count(nx: int, ny: int) -> int:
    """Number of structural + shear + bend springs of an nx-by-ny grid."""
    s = nx * (ny - 1) + ny * (nx - 1) if nx > 0 and ny > 0 else 0
    sh = 2 * max(nx - 1, 0) * max(ny - 1, 0)
    b = nx * max(ny - 2, 0) + ny * max(nx - 2, 0)
    return s + sh + b


def flat_grid(nx: int, ny: int, origin, du, dv) -> np.ndarray:
    """Rest positions origin + col*du + row*dv in FP64, shape (N,3)."""
    r, c = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    o, u, v = (np.asarray(a, dtype=np.float64) for a in (origin, du, dv))
    p = o[None, None, :] + c[..., None] * u[None, None, :] + r[..., None] * v[None, None, :]
    return p.reshape(-1, 3)


# Constants of the 32x32 reference cloth; finer cloths scale them by (h/h0)^2
# so that k/m and kd/m per node stay (within 6%) those of the 32x32 cloth and
# the 1/4800 s substep stays stable.
KS0 = (500.0, 250.0, 100.0)
KD0 = (0.5, 0.5, 0.5)
H0 = 1.0 / 31.0
DT_SUB = 1.0 / 4800.0


def scaled_constants(n: int):
    s = ((1.0 / (n - 1)) / H0) ** 2
    return tuple(k * s for k in KS0), tuple(k * s for k in KD0)


def _square_horizontal(n: int, y: float):
    h = 1.0 / (n - 1)
    return (-0.5, y, -0.5), (h, 0.0, 0.0), (0.0, 0.0, h)


def config1(steps: int = 200) -> Scene:
    """32x32 hanging cloth, two top corners pinned, +-1e-3 m jitter (seed 0),
    over a 320-triangle icosphere of radius 0.3 m centred 0.5 m below."""
    n = 32
    o, du, dv = _square_horizontal(n, 0.0)
    X0 = flat_grid(n, n, o, du, dv)
    jit = np.random.default_rng(0).uniform(-1e-3, 1e-3, (n * n, 3))
    pos = (X0 + jit).astype(np.float32)
    pinned = np.zeros(n * n, np.uint8)
    pinned[0] = pinned[n - 1] = 1
    mv, mt = sphere_mesh(2, 0.3, (0.0, -0.5, 0.0))
    return Scene("config1_32x32_L2", n, n, o, du, dv, 1.0, KS0, KD0, (0.0, -9.81, 0.0),
                 1.0 / 600.0, 8, steps, pos, np.zeros_like(pos), pinned, mv, mt)


def displaced_mesh_l6(seed: int = 0):
    """Level-6 icosphere (81,920 triangles), r = 0.4 + 0.05*noise, at origin."""
    return sphere_mesh(6, 0.4, (0.0, 0.0, 0.0), 0.05, seed)


def config2(steps: int = 1000, mesh=None) -> Scene:
    """256x256 cloth flat at y=+0.5 draped over the displaced L6 sphere."""
    n = 256
    o, du, dv = _square_horizontal(n, 0.5)
    pos = flat_grid(n, n, o, du, dv).astype(np.float32)
    ks, kd = scaled_constants(n)
    mv, mt = mesh if mesh is not None else displaced_mesh_l6(0)
    return Scene("config2_256x256_L6", n, n, o, du, dv, 1.0, ks, kd, (0.0, -9.81, 0.0),
                 1.0 / 1200.0, 4, steps, pos, np.zeros_like(pos),
                 np.zeros(n * n, np.uint8), mv, mt)


def pulling_scene(n: int = 128, mesh: str = "sphere", steps: int = 600, speed: float = 0.5) -> Scene:
    """The paper's second experiment (Section 4, Fig. 5): a cloth pulled
    across a 3D model.  n x n cloth, 1 m x 1 m, horizontal at y = 0.3 above a
    model of radius 0.25 at the origin; its leading row (z = -0.5) is pinned
    and pulled along +x at `speed` m/s (kinematic pins) while gravity drapes
    the rest over the model.  mesh: 'sphere' (5,120-triangle icosphere) or
    'l6' (the 81,920-triangle displaced mesh scaled to radius 0.25); dt 1/1200 s
    in 4 substeps."""
    o, du, dv = _square_horizontal(n, 0.3)
    pos = flat_grid(n, n, o, du, dv).astype(np.float32)
    pinned = np.zeros(n * n, np.uint8)
    pinned[:n] = 1
    ks, kd = scaled_constants(n)
    if mesh == "sphere":
        mv, mt = sphere_mesh(4, 0.25, (0.0, 0.0, 0.0))
    elif mesh == "l6":
        mv, mt = displaced_mesh_l6(0)
        mv = (mv * np.float32(0.25 / 0.45)).astype(np.float32)
    else:
        raise ValueError(mesh)
    return Scene(f"pulling_{n}x{n}_{mesh}", n, n, o, du, dv, 1.0, ks, kd, (0.0, -9.81, 0.0), 1.0 / 1200.0, 4,
                 steps, pos, np.zeros_like(pos), pinned, mv, mt, pin_velocity=(speed, 0.0, 0.0))


def wind_config3() -> Wind:
    phase = 2.0 * math.pi * float(np.random.default_rng(2).uniform())
    s = 1.0 / math.sqrt(2.0)
    return Wind(2.0, (0.0, 0.0, 1.0), (s, s, 0.0), 1.0, 2.0 * math.pi / 0.5, phase)


def config3(mesh: str = "l6", steps: int = 600, n: int = 800) -> Scene:
    """Paper-scale hanging cloth: n x n nodes in the plane z=0, top row
    pinned, gravity + seeded sinusoidal wind (2 N/kg); mesh 'none', 'l5'
    (20,480-triangle sphere r=0.25) or 'l6' (the displaced L6 mesh scaled to
    r=0.25, 81,920 triangles), centred at (0,-0.6,0.3)."""
    h = 1.0 / (n - 1)
    o, du, dv = (-0.5, 0.0, 0.0), (h, 0.0, 0.0), (0.0, -h, 0.0)
    pos = flat_grid(n, n, o, du, dv).astype(np.float32)
    pinned = np.zeros(n * n, np.uint8)
    pinned[:n] = 1
    ks, kd = scaled_constants(n)
    c = (0.0, -0.6, 0.3)
    if mesh == "none":
        mv = mt = None
    elif mesh == "l5":
        mv, mt = sphere_mesh(5, 0.25, c)
    elif mesh == "l6":
        v, f = icosphere(6)
        r = 0.4 + 0.05 * perlin_noise3(3.0 * v, 0)
        mv = ((v * r[:, None]) * (0.25 / 0.4) + np.asarray(c)[None, :]).astype(np.float32)
        mt = f.astype(np.int32)
    else:
        raise ValueError(mesh)
    return Scene(f"config3_{n}x{n}_{mesh}", n, n, o, du, dv, 1.0, ks, kd, (0.0, -9.81, 0.0),
                 1.0 / 1200.0, 4, steps, pos, np.zeros_like(pos), pinned, mv, mt,
                 wind=wind_config3())


def config4(steps: int = 256) -> Scene:
    """128x128 cloth over a 5,120-triangle icosphere (r=0.3) with per-spring
    stiffness/damping arrays (canonical spring order)."""
    n = 128
    o, du, dv = _square_horizontal(n, 0.0)
    pos = flat_grid(n, n, o, du, dv).astype(np.float32)
    ks, kd = scaled_constants(n)
    S = spring_count(n, n)
    typ = spring_types(n, n)
    ks_sp = np.asarray(ks, np.float64)[typ].astype(np.float32)
    kd_sp = np.asarray(kd, np.float64)[typ].astype(np.float32)
    assert len(ks_sp) == S
    mv, mt = sphere_mesh(4, 0.3, (0.0, -0.35, 0.0))
    pinned = np.zeros(n * n, np.uint8)
    return Scene("config4_128x128_L4", n, n, o, du, dv, 1.0, ks, kd, (0.0, -9.81, 0.0),
                 1.0 / 1200.0, 4, steps, pos, np.zeros_like(pos), pinned, mv, mt,
                 ks_spring=ks_sp, kd_spring=kd_sp)


def config4_target_ks(scene: Scene) -> np.ndarray:
    """Perturbed per-spring stiffness ks*U(0.8,1.2) (seed 3) of the target run."""
    u = np.random.default_rng(3).uniform(0.8, 1.2, len(scene.ks_spring))
    return (scene.ks_spring.astype(np.float64) * u).astype(np.float32)


# Spring directions (drow, dcol) of the canonical enumeration and their types.
SPRING_DIRS = ((0, 1), (1, 0), (1, 1), (1, -1), (0, 2), (2, 0))
SPRING_DIR_TYPE = (0, 0, 1, 1, 2, 2)


def spring_types(nx: int, ny: int) -> np.ndarray:
    """Type (0 structural, 1 shear, 2 bend) of every spring in canonical order:
    row-major nodes, each emitting the directions of SPRING_DIRS in order when
    the other end lies inside the grid.  (Input sizing only: used to lay out
    per-spring constant arrays.)"""
    out = []
    for r in range(ny):
        for c in range(nx):
            for (dr, dc), t in zip(SPRING_DIRS, SPRING_DIR_TYPE):
                if 0 <= r + dr < ny and 0 <= c + dc < nx:
                    out.append(t)
    return np.asarray(out, dtype=np.int64)


def config5(count: int = 256, steps: int = 500) -> List[Scene]:
    """Batch of independent cloths: side ~ round(exp(U(ln16, ln512))) and a
    displaced icosphere of level L in {3,4,5,6} each (seed 1)."""
    rng = np.random.default_rng(1)
    sides = np.rint(np.exp(rng.uniform(math.log(16), math.log(512), count))).astype(int)
    levels = rng.integers(3, 7, count)
    out = []
    for i in range(count):
        n = int(sides[i])
        o, du, dv = _square_horizontal(n, 0.5)
        pos = flat_grid(n, n, o, du, dv).astype(np.float32)
        ks, kd = scaled_constants(n)
        mv, mt = sphere_mesh(int(levels[i]), 0.4, (0.0, 0.0, 0.0), 0.05, 1000 + i)
        out.append(Scene(f"config5_{i}_{n}x{n}_L{levels[i]}", n, n, o, du, dv, 1.0, ks, kd,
                         (0.0, -9.81, 0.0), 1.0 / 1200.0, 10, steps, pos, np.zeros_like(pos),
                         np.zeros(n * n, np.uint8), mv, mt))
    return out


def small_collision_scene(n: int = 24, level: int = 2, gap: float = 0.01, seed: int = 5,
                          substeps: int = 4, dt: float = 1.0 / 1200.0) -> Scene:
    """A cloth that starts ``gap`` metres above the highest vertex of an
    icosphere of radius 0.3 with a downward velocity, so that contacts begin within a few steps
    (parity cases that exercise the collision response early)."""
    mv, mt = sphere_mesh(level, 0.3, (0.0, 0.0, 0.0))
    o, du, dv = _square_horizontal(n, float(mv[:, 1].max()) + gap)
    X0 = flat_grid(n, n, o, du, dv)
    jit = np.random.default_rng(seed).uniform(-2e-4, 2e-4, (n * n, 3))
    pos = (X0 + jit).astype(np.float32)
    vel = np.zeros_like(pos)
    vel[:, 1] = -1.0
    ks, kd = scaled_constants(n)
    return Scene(f"contact_{n}x{n}_L{level}", n, n, o, du, dv, 1.0, ks, kd, (0.0, -9.81, 0.0),
                 dt, substeps, 100, pos, vel, np.zeros(n * n, np.uint8), mv, mt)
