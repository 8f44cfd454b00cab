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


# ------------------------------------------------ config-4 segment gradients

def config4_target(oracle):
    """The target state of the differentiation workload: the FP64 run with
    per-spring ks * U(0.8, 1.2) (seed 3) after 256 steps."""
    sc = cs.config4()
    grid = oracle.Grid(sc.mesh_verts, sc.mesh_tris)
    cl = oracle.Cloth(sc, ks_spring=cs.config4_target_ks(sc).astype(np.float64),
                      kd_spring=sc.kd_spring.astype(np.float64))
    tgt, _ = oracle.step(cl, sc.init_pos, sc.init_vel, 0, sc.steps * sc.substeps, grid)
    return tgt


def segment_final(args):
    """Final FP64 oracle positions and contact signature of a config-4 segment
    from a given state (worker of a spawned process pool)."""
    import oracle
    x0, v0, ks, kd, k0, nsub = args
    sc = cs.config4()
    grid = oracle.Grid(sc.mesh_verts, sc.mesh_tris)
    cl = oracle.Cloth(sc, ks_spring=ks, kd_spring=kd)
    x, _, sig = oracle.step_signature(cl, x0, v0, k0, nsub, grid)
    return x, sig


def f32_segment_grads(x0, v0, k0, nsub, tgt):
    """Gradients of the config-4 segment loss from the float32 restatement of
    the oracle (oracle.f32): (ks, kd, v0, final positions)."""
    import oracle.f32 as o32
    sc = cs.config4()
    grid = o32.Grid(sc.mesh_verts, sc.mesh_tris)
    cl = o32.Cloth(sc, ks_spring=sc.ks_spring, kd_spring=sc.kd_spring)
    x, _ = o32.step(cl, x0, v0, k0, nsub, grid)
    lx = (2.0 * (x.astype(np.float64) - tgt) / sc.n).astype(np.float32)
    _, lv0, gks, gkd = o32.adjoint(cl, x0, v0, k0, nsub, lx, np.zeros_like(lx), grid)
    return gks, gkd, lv0, x


def config4_segment_fd(x0, v0, k0, nsub, tgt, grads, seed, nkeep=32, ncand=64, h=1e-6, workers=16):
    """FP64 central differences of the config-4 segment loss (mean squared
    distance of the final positions to ``tgt``) from the state (x0, v0) at
    global substep k0, over ``nkeep`` seeded parameters (ks or kd of one
    spring, or one component of one initial velocity).  A candidate is
    re-drawn when its +-h or +-h/10 runs change the contact set or the active
    hits, or when the two quotients disagree by more than 1e-3 (relative,
    floored like the metric).

    grads: {name: (gks, gkd, gv0)}.  Returns ({name: rel err over the kept
    parameters}, kept [(kind, idx)], fd values, re-drawn list), rel err =
    |g - g_fd| / max(|g_fd|, 1e-3 max_k |g_fd,k|)."""
    import multiprocessing as mp
    sc = cs.config4()
    ks = sc.ks_spring.astype(np.float64)
    kd = sc.kd_spring.astype(np.float64)
    x0 = np.asarray(x0, np.float64)
    v0 = np.asarray(v0, np.float64)
    rng = np.random.default_rng(seed)

    def perturbed(kind, idx, hh):
        if kind == "v0":
            i, c = idx
            vp, vm = v0.copy(), v0.copy()
            vp[i, c] += hh
            vm[i, c] -= hh
            return [(x0, vp, ks, kd, k0, nsub), (x0, vm, ks, kd, k0, nsub)]
        base = ks if kind == "ks" else kd
        p, m = base.copy(), base.copy()
        p[idx] += hh
        m[idx] -= hh
        if kind == "ks":
            return [(x0, v0, p, kd, k0, nsub), (x0, v0, m, kd, k0, nsub)]
        return [(x0, v0, ks, p, k0, nsub), (x0, v0, ks, m, k0, nsub)]

    jobs, cands = [(x0, v0, ks, kd, k0, nsub)], []
    for _ in range(ncand):
        kind = ("ks", "kd", "v0")[int(rng.integers(3))]
        idx = (int(rng.integers(sc.n)), int(rng.integers(3))) if kind == "v0" else int(rng.integers(len(ks)))
        cands.append((kind, idx))
        jobs += perturbed(kind, idx, h) + perturbed(kind, idx, h / 10)
    with mp.get_context("spawn").Pool(min(workers, max(2, mp.cpu_count() or 2))) as pool:
        res = pool.map(segment_final, jobs)
    sig0 = res[0][1]

    def quotient(a, b, hh):
        (xp, sp), (xm, sm) = a, b
        dL = float(np.sum((xp - xm) * (xp + xm - 2.0 * tgt)) / len(xp))
        return dL / (2.0 * hh), sp == sig0 and sm == sig0

    rows = []
    for j, (kind, idx) in enumerate(cands):
        f1, ok1 = quotient(res[1 + 4 * j], res[2 + 4 * j], h)
        f2, ok2 = quotient(res[3 + 4 * j], res[4 + 4 * j], h / 10)
        rows.append((kind, idx, f1, f2, ok1 and ok2))
    same = [r for r in rows if r[4]]
    assert len(same) >= nkeep
    floor = 1e-3 * max(abs(r[2]) for r in same[:nkeep])
    kept, fds, redrawn = [], [], []
    for kind, idx, f1, f2, ok in rows:
        if not ok or abs(f1 - f2) > 1e-3 * max(abs(f1), floor):
            redrawn.append((kind, idx))
            continue
        kept.append((kind, idx))
        fds.append(f1)
        if len(kept) == nkeep:
            break
    assert len(kept) == nkeep
    fds = np.array(fds)
    rel = {}
    for name, (gks, gkd, gv0) in grads.items():
        src = {"ks": np.asarray(gks), "kd": np.asarray(gkd), "v0": np.asarray(gv0).reshape(-1, 3)}
        g = np.array([float(src[kind][idx]) for kind, idx in kept])
        rel[name] = np.abs(g - fds) / np.maximum(np.abs(fds), floor)
    return rel, kept, fds, redrawn
