"""Small scene builders and independent geometry checks shared by the tests."""
from __future__ import annotations

import os

import numpy as np

import cloth_scenes as cs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def make_scene(nx, ny, *, origin=(0.0, 0.0, 0.0), du=(0.1, 0.0, 0.0), dv=(0.0, 0.0, 0.1),
               total_mass=1.0, ks=(0.0, 0.0, 0.0), kd=(0.0, 0.0, 0.0), gravity=(0.0, 0.0, 0.0),
               dt=1e-3, substeps=1, pos=None, vel=None, pinned=None, mesh=None,
               wind=None, delta=1e-4, eps=1e-7, t_min=0.0, restitution=-0.5, name="custom"):
    N = nx * ny
    if pos is None:
        pos = cs.flat_grid(nx, ny, origin, du, dv)
    pos = np.asarray(pos, dtype=np.float32).reshape(N, 3)
    vel = np.zeros((N, 3), np.float32) if vel is None else np.asarray(vel, np.float32).reshape(N, 3)
    pinned = np.zeros(N, np.uint8) if pinned is None else np.asarray(pinned, np.uint8)
    mv, mt = (None, None) if mesh is None else mesh
    return cs.Scene(name, nx, ny, tuple(origin), tuple(du), tuple(dv), total_mass, tuple(ks), tuple(kd),
                    tuple(gravity), dt, substeps, 1, pos, vel, pinned, mv, mt,
                    contact_offset=delta, mt_eps=eps, mt_t_min=t_min, restitution=restitution,
                    wind=wind if wind is not None else cs.Wind())


def floor_mesh():
    """Square [0,1]x{0}x[0,1], two triangles split along the x=z diagonal."""
    v = np.array([[0, 0, 0], [1, 0, 0], [1, 0, 1], [0, 0, 1]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return v, t


def stencil_pairs(nx, ny):
    """All node pairs (i<j) at a structural, shear or bend offset, by brute
    force over every pair of nodes (independent of the canonical order)."""
    offs = {(0, 1), (1, 0), (1, 1), (1, -1), (0, 2), (2, 0)}
    offs |= {(-a, -b) for a, b in offs}
    out = set()
    N = nx * ny
    for i in range(N):
        for j in range(i + 1, N):
            dr, dc = j // nx - i // nx, j % nx - i % nx
            if (dr, dc) in offs:
                out.add((i, j))
    return out


def spring_energy(nx, ny, X0, x, ks_of_pair):
    """Elastic energy sum 1/2 k (|x_j - x_i| - |X0_j - X0_i|)^2 over pairs."""
    E = 0.0
    for (i, j) in stencil_pairs(nx, ny):
        L0 = np.linalg.norm(X0[j] - X0[i])
        L = np.linalg.norm(x[j] - x[i])
        E += 0.5 * ks_of_pair(i, j) * (L - L0) ** 2
    return E


def pair_type(nx, i, j):
    dr, dc = abs(j // nx - i // nx), abs(j % nx - i % nx)
    if dr + dc == 1:
        return 0
    if dr == 1 and dc == 1:
        return 1
    return 2


def ray_parity_inside(points, verts, tris, direction=(0.5773502691896258, 0.5773502691896258, 0.5773502691896258)):
    """Point-in-closed-mesh test by counting crossings of a ray (FP64)."""
    V = np.asarray(verts, np.float64)
    T = np.asarray(tris, np.int64)
    A, B, Cc = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    e1, e2 = B - A, Cc - A
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    inside = np.zeros(len(points), bool)
    for k, p in enumerate(np.asarray(points, np.float64)):
        h = np.cross(d, e2)
        a = np.einsum("ij,ij->i", e1, h)
        ok = np.abs(a) > 1e-15
        f = np.where(ok, 1.0 / np.where(ok, a, 1.0), 0.0)
        s = p - A
        u = f * np.einsum("ij,ij->i", s, h)
        q = np.cross(s, e1)
        v = f * (q @ d)
        t = f * np.einsum("ij,ij->i", e2, q)
        hit = ok & (u >= 0) & (u <= 1) & (v >= 0) & (u + v <= 1) & (t > 0)
        inside[k] = (int(hit.sum()) % 2) == 1
    return inside
