"""FP64 CPU oracle of the mass-spring cloth step (arXiv 2507.11794).

TEST INFRASTRUCTURE ONLY.  The product path never imports this package: only
the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of the
benchmark may load it.  The arithmetic lives in ``oracle.c`` (plain C, double
precision, one thread); this module compiles it with gcc and marshals numpy
arrays through ctypes.  It shares no code with the CUDA library.

Functions (each cites the passage of the paper it follows, see oracle.c):

* ``springs``        canonical spring enumeration (Algorithm 1's Springs buffer)
* ``spring_forces``  Algorithm 1 in double, spring-centric accumulation
* ``accel``          F/m + gravity + wind (Section 3, Euler step inputs)
* ``mt``             extended Moller-Trumbore test (Section 3)
* ``Grid``           uniform grid over the surface triangles (broad phase,
                     float32 cell formula; not in the paper, which tests all pairs)
* ``step``           full substeps: forces, symplectic Euler, collision, the
                     Algorithm 2 response
* ``adjoint``        reverse mode of ``step`` with the contact set frozen:
                     gradients w.r.t. final-state adjoints of the initial state and
                     of per-spring ks, kd (not in the paper)
* ``step_edges``     the paper's own narrow phase: cloth-triangle edges at the
                     updated positions against the surface triangles
* ``grid_triangles`` / ``normals``  the cloth grid's triangle list and its
                     per-vertex normals, the update that precedes rendering
                     (Section 3); plain numpy in double
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OcCloth(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("origin", C.c_double * 3), ("du", C.c_double * 3), ("dv", C.c_double * 3),
        ("mass", C.c_double),
        ("ks", C.c_double * 3), ("kd", C.c_double * 3),
        ("ks_spring", C.POINTER(C.c_double)), ("kd_spring", C.POINTER(C.c_double)),
        ("pinned", C.POINTER(C.c_uint8)),
        ("gravity", C.c_double * 3),
        ("dt_s", C.c_double),
        ("delta", C.c_double), ("eps", C.c_double), ("t_min", C.c_double), ("restitution", C.c_double),
        ("wind_amp", C.c_double), ("wind_dir", C.c_double * 3), ("wind_udir", C.c_double * 3),
        ("wind_freq", C.c_double), ("wind_kappa", C.c_double), ("wind_phase", C.c_double),
        ("pin_vel", C.c_double * 3),
    ]


class OcGrid(C.Structure):
    _fields_ = [
        ("h", C.c_float), ("inv", C.c_float), ("origin", C.c_float * 3),
        ("dims", C.c_int32 * 3), ("ncells", C.c_int64), ("nentries", C.c_int64),
        ("cell_start", C.POINTER(C.c_int32)), ("tri_ids", C.POINTER(C.c_int32)),
    ]


class OcMesh(C.Structure):
    _fields_ = [("verts", C.POINTER(C.c_float)), ("nverts", C.c_int32),
                ("tris", C.POINTER(C.c_int32)), ("ntris", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, fp, ip = C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_int32)
            L.oc_springs.argtypes = [C.c_int32, C.c_int32, ip, ip, ip, C.c_int64]
            L.oc_springs.restype = C.c_int64
            L.oc_spring_forces.argtypes = [C.POINTER(OcCloth), dp, dp, dp]
            L.oc_accel.argtypes = [C.POINTER(OcCloth), dp, dp, C.c_double, dp]
            L.oc_mt.argtypes = [dp, dp, dp, dp, dp, C.c_double, C.c_double, dp]
            L.oc_mt.restype = C.c_int
            L.oc_grid_build.argtypes = [fp, C.c_int32, ip, C.c_int32, C.POINTER(OcGrid)]
            L.oc_grid_build.restype = C.c_int
            L.oc_grid_free.argtypes = [C.POINTER(OcGrid)]
            L.oc_candidates_f32.argtypes = [C.POINTER(OcGrid), fp, fp, ip, C.c_int64]
            L.oc_candidates_f32.restype = C.c_int64
            L.oc_step.argtypes = [C.POINTER(OcCloth), C.POINTER(OcMesh), C.POINTER(OcGrid),
                                  dp, dp, C.c_int64, C.c_int32, ip]
            L.oc_step.restype = C.c_int
            L.oc_step_ex.argtypes = [C.POINTER(OcCloth), C.POINTER(OcMesh), C.POINTER(OcGrid), dp, dp, C.c_int64,
                                     C.c_int32, ip, dp, dp, dp, C.POINTER(C.c_uint64)]
            L.oc_step_ex.restype = C.c_int
            L.oc_step_edges.argtypes = [C.POINTER(OcCloth), C.POINTER(OcMesh), C.POINTER(OcGrid),
                                        dp, dp, C.c_int64, C.c_int32, ip]
            L.oc_step_edges.restype = C.c_int
            L.oc_edge_affected.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, ip]
            L.oc_edge_affected.restype = C.c_int32
            L.oc_adjoint.argtypes = [C.POINTER(OcCloth), C.POINTER(OcMesh), C.POINTER(OcGrid), dp, dp, C.c_int64,
                                     C.c_int32, dp, dp, dp, dp]
            L.oc_adjoint.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class Cloth:
    """Double-precision parameter block of one cloth (from a scene)."""

    def __init__(self, scene, ks_spring=None, kd_spring=None):
        self.scene = scene
        s = scene
        self.N = s.nx * s.ny
        c = OcCloth()
        c.nx, c.ny = s.nx, s.ny
        for k in range(3):
            c.origin[k], c.du[k], c.dv[k] = float(s.origin[k]), float(s.du[k]), float(s.dv[k])
            c.ks[k], c.kd[k] = float(s.ks[k]), float(s.kd[k])
            c.gravity[k] = float(s.gravity[k])
            c.wind_dir[k], c.wind_udir[k] = float(s.wind.dir[k]), float(s.wind.udir[k])
        c.mass = float(s.total_mass) / self.N
        ks_sp = ks_spring if ks_spring is not None else s.ks_spring
        kd_sp = kd_spring if kd_spring is not None else s.kd_spring
        self._ks = None if ks_sp is None else np.ascontiguousarray(ks_sp, dtype=np.float64)
        self._kd = None if kd_sp is None else np.ascontiguousarray(kd_sp, dtype=np.float64)
        c.ks_spring = _ptr(self._ks, C.c_double) if self._ks is not None else None
        c.kd_spring = _ptr(self._kd, C.c_double) if self._kd is not None else None
        self._pin = np.ascontiguousarray(s.pinned, dtype=np.uint8)
        c.pinned = _ptr(self._pin, C.c_uint8)
        c.dt_s = float(s.dt) / int(s.substeps)
        c.delta, c.eps, c.restitution = float(s.contact_offset), float(s.mt_eps), float(s.restitution)
        c.t_min = float(s.mt_t_min)
        c.wind_amp, c.wind_freq = float(s.wind.amp), float(s.wind.freq)
        c.wind_kappa, c.wind_phase = float(s.wind.kappa), float(s.wind.phase)
        for k in range(3):
            c.pin_vel[k] = float(getattr(s, "pin_velocity", (0.0, 0.0, 0.0))[k])
        self.c = c


class Grid:
    """The oracle's own uniform grid over a float32 mesh."""

    def __init__(self, verts, tris):
        self.verts = np.ascontiguousarray(verts, dtype=np.float32)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.g = OcGrid()
        rc = lib().oc_grid_build(_ptr(self.verts, C.c_float), len(self.verts),
                                 _ptr(self.tris, C.c_int32), len(self.tris), C.byref(self.g))
        if rc != 0:
            lib().oc_grid_free(C.byref(self.g))
            raise ValueError(f"oc_grid_build failed ({rc})")
        self.mesh = OcMesh(_ptr(self.verts, C.c_float), len(self.verts),
                           _ptr(self.tris, C.c_int32), len(self.tris))

    def __del__(self):
        try:
            lib().oc_grid_free(C.byref(self.g))
        except Exception:
            pass

    @property
    def params(self):
        g = self.g
        return dict(h=g.h, inv=g.inv, origin=tuple(g.origin), dims=tuple(g.dims),
                    ncells=g.ncells, nentries=g.nentries)

    def cell_start(self):
        return np.ctypeslib.as_array(self.g.cell_start, shape=(self.g.ncells + 1,)).copy()

    def tri_ids(self):
        if self.g.nentries == 0:
            return np.zeros(0, np.int32)
        return np.ctypeslib.as_array(self.g.tri_ids, shape=(self.g.nentries,)).copy()

    def candidates_f32(self, S, E):
        S = np.ascontiguousarray(S, dtype=np.float32)
        E = np.ascontiguousarray(E, dtype=np.float32)
        cap = 256
        while True:
            out = np.empty(cap, np.int32)
            n = lib().oc_candidates_f32(C.byref(self.g), _ptr(S, C.c_float), _ptr(E, C.c_float),
                                        _ptr(out, C.c_int32), cap)
            if n <= cap:
                return out[:n].copy()
            cap = int(n)


def springs(nx, ny):
    """(a, b, type) int32 arrays of the canonical spring enumeration."""
    S = lib().oc_springs(nx, ny, None, None, None, 0)
    a, b, t = (np.empty(S, np.int32) for _ in range(3))
    lib().oc_springs(nx, ny, _ptr(a, C.c_int32), _ptr(b, C.c_int32), _ptr(t, C.c_int32), S)
    return a, b, t


def spring_forces(cloth: Cloth, x, v):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    F = np.empty_like(x)
    lib().oc_spring_forces(C.byref(cloth.c), _ptr(x, C.c_double), _ptr(v, C.c_double), _ptr(F, C.c_double))
    return F.reshape(-1, 3)


def accel(cloth: Cloth, x, v, t):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    A = np.empty_like(x)
    lib().oc_accel(C.byref(cloth.c), _ptr(x, C.c_double), _ptr(v, C.c_double), float(t), _ptr(A, C.c_double))
    return A.reshape(-1, 3)


def mt(S, E, V0, V1, V2, eps=1e-7, t_min=None):
    """Extended Moller-Trumbore test; returns t on a hit, else None.
    t_min defaults to eps (the paper's literal bound eps < t)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (S, E, V0, V1, V2)]
    t = C.c_double(0.0)
    tm = float(eps) if t_min is None else float(t_min)
    hit = lib().oc_mt(*[_ptr(a, C.c_double) for a in arrs], float(eps), tm, C.byref(t))
    return t.value if hit else None


def step(cloth: Cloth, x, v, k0: int, nsub: int, grid: Grid | None = None, brute: bool = False,
         want_hits: bool = False):
    """Advance ``nsub`` substeps from global substep ``k0`` (in place on copies).

    grid: the oracle Grid of the scene's mesh (None = no collision unless
    ``brute``); brute=True tests every triangle (needs grid for the mesh
    arrays only).  Returns (x, v) or (x, v, hits).
    """
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1).copy()
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1).copy()
    hits = np.zeros(cloth.N, np.int32)
    mesh = C.byref(grid.mesh) if grid is not None else None
    g = C.byref(grid.g) if (grid is not None and not brute) else None
    rc = lib().oc_step(C.byref(cloth.c), mesh, g, _ptr(x, C.c_double), _ptr(v, C.c_double),
                       int(k0), int(nsub), _ptr(hits, C.c_int32))
    if rc != 0:
        raise RuntimeError(f"oc_step failed ({rc})")
    if want_hits:
        return x.reshape(-1, 3), v.reshape(-1, 3), hits
    return x.reshape(-1, 3), v.reshape(-1, 3)


def step_edges(cloth: Cloth, x, v, k0: int, nsub: int, grid: Grid | None = None, brute: bool = False,
               want_hits: bool = False):
    """Like ``step`` with the paper's edge-triangle narrow phase: the cloth
    triangulation's edges at the updated positions against the surface
    triangles, every vertex of the triangles sharing a hit edge moved from
    its previous position towards the hit point (stopping delta short),
    averaged over its hits.  hits: per node, the hits it received."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1).copy()
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1).copy()
    hits = np.zeros(cloth.N, np.int32)
    mesh = C.byref(grid.mesh) if grid is not None else None
    g = C.byref(grid.g) if (grid is not None and not brute) else None
    rc = lib().oc_step_edges(C.byref(cloth.c), mesh, g, _ptr(x, C.c_double), _ptr(v, C.c_double),
                             int(k0), int(nsub), _ptr(hits, C.c_int32))
    if rc != 0:
        raise RuntimeError(f"oc_step_edges failed ({rc})")
    if want_hits:
        return x.reshape(-1, 3), v.reshape(-1, 3), hits
    return x.reshape(-1, 3), v.reshape(-1, 3)


def edge_affected(nx: int, ny: int, r: int, c: int, q: int):
    """Nodes affected by a hit on edge kind q (0 right, 1 down, 2 diagonal)
    owned by node (r, c): the vertices of the cloth triangles containing it."""
    out = np.zeros(4, np.int32)
    n = lib().oc_edge_affected(nx, ny, r, c, q, _ptr(out, C.c_int32))
    return sorted(int(a) for a in out[:n])


def run(scene, steps: int, grid: Grid | None = None, x=None, v=None, k0: int = 0):
    """Run ``steps`` outer steps of ``scene`` from its initial (float32) state."""
    cl = Cloth(scene)
    if grid is None and scene.mesh_tris is not None and len(scene.mesh_tris):
        grid = Grid(scene.mesh_verts, scene.mesh_tris)
    x = scene.init_pos if x is None else x
    v = scene.init_vel if v is None else v
    return step(cl, x, v, k0, steps * scene.substeps, grid)


def step_signature(cloth: Cloth, x, v, k0: int, nsub: int, grid: Grid | None = None):
    """Like ``step`` (grid broad phase) but also returns a 64-bit signature of
    every (substep, node, hit triangle, t > delta): equal signatures mean the
    same contact sets with the same active hits."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1).copy()
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1).copy()
    sig = C.c_uint64(0xcbf29ce484222325)
    mesh = C.byref(grid.mesh) if grid is not None else None
    g = C.byref(grid.g) if grid is not None else None
    rc = lib().oc_step_ex(C.byref(cloth.c), mesh, g, _ptr(x, C.c_double), _ptr(v, C.c_double), int(k0), int(nsub),
                          None, None, None, None, C.byref(sig))
    if rc != 0:
        raise RuntimeError(f"oc_step_ex failed ({rc})")
    return x.reshape(-1, 3), v.reshape(-1, 3), sig.value


def adjoint(cloth: Cloth, x0, v0, k0: int, nsub: int, lx, lv, grid: Grid | None = None):
    """Reverse mode of ``nsub`` substeps from (x0, v0): given dL/dx, dL/dv at
    the end returns (dL/dx0, dL/dv0, dL/dks, dL/dkd), the last two per spring
    in canonical order (zeros when the cloth has no per-spring arrays is not
    special: they are the gradients w.r.t. each spring's constants)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1)
    v0 = np.ascontiguousarray(v0, dtype=np.float64).reshape(-1)
    lx = np.ascontiguousarray(lx, dtype=np.float64).reshape(-1).copy()
    lv = np.ascontiguousarray(lv, dtype=np.float64).reshape(-1).copy()
    S = lib().oc_springs(cloth.c.nx, cloth.c.ny, None, None, None, 0)
    gks = np.zeros(S, np.float64)
    gkd = np.zeros(S, np.float64)
    mesh = C.byref(grid.mesh) if grid is not None else None
    g = C.byref(grid.g) if grid is not None else None
    rc = lib().oc_adjoint(C.byref(cloth.c), mesh, g, _ptr(x0, C.c_double), _ptr(v0, C.c_double), int(k0),
                          int(nsub), _ptr(lx, C.c_double), _ptr(lv, C.c_double), _ptr(gks, C.c_double),
                          _ptr(gkd, C.c_double))
    if rc != 0:
        raise RuntimeError(f"oc_adjoint failed ({rc})")
    return lx.reshape(-1, 3), lv.reshape(-1, 3), gks, gkd


# ---------------------------------------------------------------- normals
# Section 3 ends a frame with a normal vector update before rendering.  The
# paper does not give the formula; the reading here: each grid quad
# (r, c), (r, c+1), (r+1, c), (r+1, c+1) is split along its (r, c)-(r+1, c+1)
# diagonal into (r,c)-(r+1,c)-(r+1,c+1) and (r,c)-(r+1,c+1)-(r,c+1); a vertex
# normal is the normalised sum of the unnormalised face normals
# (e1 x e2, so larger faces weigh more) of the triangles that contain it, and
# the zero vector where that sum is zero.

def grid_triangles(nx: int, ny: int) -> np.ndarray:
    """Triangles of the cloth grid, [2 (nx-1)(ny-1), 3] node indices, quad by
    quad in row-major order, two per quad as described above."""
    tris = []
    for r in range(ny - 1):
        for c in range(nx - 1):
            a, b = r * nx + c, r * nx + c + 1
            d, e = (r + 1) * nx + c, (r + 1) * nx + c + 1
            tris.append((a, d, e))
            tris.append((a, e, b))
    return np.asarray(tris, dtype=np.int64).reshape(-1, 3)


def normals(pos, nx: int, ny: int) -> np.ndarray:
    """Per-vertex normals [N, 3] (double) of the cloth state pos [N, 3]."""
    x = np.asarray(pos, dtype=np.float64).reshape(nx * ny, 3)
    acc = np.zeros_like(x)
    for a, b, c in grid_triangles(nx, ny):
        n = np.cross(x[b] - x[a], x[c] - x[a])
        acc[a] += n
        acc[b] += n
        acc[c] += n
    out = np.zeros_like(acc)
    ln = np.linalg.norm(acc, axis=1)
    ok = ln > 0.0
    out[ok] = acc[ok] / ln[ok, None]
    return out
