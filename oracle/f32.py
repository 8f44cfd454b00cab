"""Float32 restatement of the oracle: the precision floor of the method.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the product path
never imports it.  It answers one question the FP64 oracle cannot: how close
can ANY float32 evaluation of the step and of its adjoint come to FP64 finite
differences?  The C source is ``oracle.c`` itself with the type ``double``
replaced by ``float`` (a token substitution made at build time), its math
calls by their float forms (``sqrtf``, ``fabsf``, ``floorf``, ``sinf``) and
its floating constants compiled single precision
(``-fsingle-precision-constant``), so it takes the same steps in the same
order with every intermediate rounded to float32.  Nothing of the CUDA path
is used; the tests compare the GPU's float32 gradients with the errors this
restatement makes on the same inputs.

Only what those comparisons need is wrapped: ``Cloth``, ``Grid``, ``step``
and ``adjoint``, with the signatures of the FP64 module's functions and
float32 arrays in and out.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle_f32.so")
_lock = threading.Lock()
_lib = None

_MATH = {"sqrt": "sqrtf", "fabs": "fabsf", "floor": "floorf", "sin": "sinf"}


def restated_source() -> str:
    """oracle.c with every ``double`` declared ``float`` and float math calls."""
    with open(_SRC) as f:
        src = f.read()
    src = re.sub(r"\bdouble\b", "float", src)
    for d, s in _MATH.items():
        src = re.sub(r"\b%s\(" % d, s + "(", src)
    return src


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                                                          os.path.getmtime(__file__)):
        with tempfile.TemporaryDirectory() as td:
            c = os.path.join(td, "oracle_f32.c")
            with open(c, "w") as f:
                f.write(restated_source())
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                                   "-fsingle-precision-constant", "-fexcess-precision=standard", "-I", _HERE,
                                   "-fPIC", "-shared", "-o", tmp, c, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class OcCloth(C.Structure):
    # the FP64 module's OcCloth with every double field float
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("origin", C.c_float * 3), ("du", C.c_float * 3), ("dv", C.c_float * 3),
        ("mass", C.c_float),
        ("ks", C.c_float * 3), ("kd", C.c_float * 3),
        ("ks_spring", C.POINTER(C.c_float)), ("kd_spring", C.POINTER(C.c_float)),
        ("pinned", C.POINTER(C.c_uint8)),
        ("gravity", C.c_float * 3),
        ("dt_s", C.c_float),
        ("delta", C.c_float), ("eps", C.c_float), ("t_min", C.c_float), ("restitution", C.c_float),
        ("wind_amp", C.c_float), ("wind_dir", C.c_float * 3), ("wind_udir", C.c_float * 3),
        ("wind_freq", C.c_float), ("wind_kappa", C.c_float), ("wind_phase", C.c_float),
        ("pin_vel", C.c_float * 3),
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
            fp, ip = C.POINTER(C.c_float), C.POINTER(C.c_int32)
            L.oc_springs.argtypes = [C.c_int32, C.c_int32, ip, ip, ip, C.c_int64]
            L.oc_springs.restype = C.c_int64
            L.oc_grid_build.argtypes = [fp, C.c_int32, ip, C.c_int32, C.POINTER(OcGrid)]
            L.oc_grid_build.restype = C.c_int
            L.oc_grid_free.argtypes = [C.POINTER(OcGrid)]
            L.oc_step.argtypes = [C.POINTER(OcCloth), C.POINTER(OcMesh), C.POINTER(OcGrid),
                                  fp, fp, C.c_int64, C.c_int32, ip]
            L.oc_step.restype = C.c_int
            L.oc_adjoint.argtypes = [C.POINTER(OcCloth), C.POINTER(OcMesh), C.POINTER(OcGrid), fp, fp, C.c_int64,
                                     C.c_int32, fp, fp, fp, fp]
            L.oc_adjoint.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32).reshape(-1).copy()


class Cloth:
    """Float32 parameter block of one cloth (from a scene)."""

    def __init__(self, scene, ks_spring=None, kd_spring=None):
        s = scene
        self.N = s.nx * s.ny
        c = OcCloth()
        c.nx, c.ny = s.nx, s.ny
        for k in range(3):
            c.origin[k], c.du[k], c.dv[k] = float(s.origin[k]), float(s.du[k]), float(s.dv[k])
            c.ks[k], c.kd[k] = float(s.ks[k]), float(s.kd[k])
            c.gravity[k] = float(s.gravity[k])
            c.wind_dir[k], c.wind_udir[k] = float(s.wind.dir[k]), float(s.wind.udir[k])
            c.pin_vel[k] = float(getattr(s, "pin_velocity", (0.0, 0.0, 0.0))[k])
        c.mass = np.float32(s.total_mass) / np.float32(self.N)
        ks_sp = ks_spring if ks_spring is not None else s.ks_spring
        kd_sp = kd_spring if kd_spring is not None else s.kd_spring
        self._ks = None if ks_sp is None else _f32(ks_sp)
        self._kd = None if kd_sp is None else _f32(kd_sp)
        c.ks_spring = _ptr(self._ks) if self._ks is not None else None
        c.kd_spring = _ptr(self._kd) if self._kd is not None else None
        self._pin = np.ascontiguousarray(s.pinned, dtype=np.uint8)
        c.pinned = self._pin.ctypes.data_as(C.POINTER(C.c_uint8))
        c.dt_s = np.float32(s.dt) / np.float32(s.substeps)
        c.delta, c.eps, c.restitution = float(s.contact_offset), float(s.mt_eps), float(s.restitution)
        c.t_min = float(s.mt_t_min)
        c.wind_amp, c.wind_freq = float(s.wind.amp), float(s.wind.freq)
        c.wind_kappa, c.wind_phase = float(s.wind.kappa), float(s.wind.phase)
        self.c = c


class Grid:
    """The restatement's uniform grid over a float32 mesh."""

    def __init__(self, verts, tris):
        self.verts = np.ascontiguousarray(verts, dtype=np.float32)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.g = OcGrid()
        ip = C.POINTER(C.c_int32)
        rc = lib().oc_grid_build(_ptr(self.verts), len(self.verts), self.tris.ctypes.data_as(ip), len(self.tris),
                                 C.byref(self.g))
        if rc != 0:
            lib().oc_grid_free(C.byref(self.g))
            raise ValueError(f"oc_grid_build failed ({rc})")
        self.mesh = OcMesh(_ptr(self.verts), len(self.verts), self.tris.ctypes.data_as(ip), len(self.tris))

    def __del__(self):
        try:
            lib().oc_grid_free(C.byref(self.g))
        except Exception:
            pass


def step(cloth: Cloth, x, v, k0: int, nsub: int, grid: Grid | None = None):
    """``nsub`` substeps from global substep ``k0`` in float32: (x, v)."""
    x, v = _f32(x), _f32(v)
    hits = np.zeros(cloth.N, np.int32)
    mesh = C.byref(grid.mesh) if grid is not None else None
    g = C.byref(grid.g) if grid is not None else None
    rc = lib().oc_step(C.byref(cloth.c), mesh, g, _ptr(x), _ptr(v), int(k0), int(nsub),
                       hits.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc != 0:
        raise RuntimeError(f"oc_step failed ({rc})")
    return x.reshape(-1, 3), v.reshape(-1, 3)


def adjoint(cloth: Cloth, x0, v0, k0: int, nsub: int, lx, lv, grid: Grid | None = None):
    """Reverse mode in float32: (dL/dx0, dL/dv0, dL/dks, dL/dkd)."""
    x0, v0, lx, lv = _f32(x0), _f32(v0), _f32(lx), _f32(lv)
    S = lib().oc_springs(cloth.c.nx, cloth.c.ny, None, None, None, 0)
    gks = np.zeros(S, np.float32)
    gkd = np.zeros(S, np.float32)
    mesh = C.byref(grid.mesh) if grid is not None else None
    g = C.byref(grid.g) if grid is not None else None
    rc = lib().oc_adjoint(C.byref(cloth.c), mesh, g, _ptr(x0), _ptr(v0), int(k0), int(nsub), _ptr(lx), _ptr(lv),
                          _ptr(gks), _ptr(gkd))
    if rc != 0:
        raise RuntimeError(f"oc_adjoint failed ({rc})")
    return lx.reshape(-1, 3), lv.reshape(-1, 3), gks, gkd
