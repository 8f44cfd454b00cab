"""ctypes binding of libcloth.so (the C ABI of include/cloth.h).

Argument marshalling only: every step of the cloth path runs in the CUDA
kernels of the library.  The functions keep the C names (cloth_create,
cloth_set_mesh, cloth_step, cloth_read, cloth_destroy, ...) and raise
``ClothError`` on a negative status.  If the library is missing or cannot be
loaded, ``lib()`` raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcloth.so")

CLOTH_OK = 0
CLOTH_ERR_INVALID_ARG = -1
CLOTH_ERR_OOM = -2
CLOTH_ERR_CUDA = -3
CLOTH_ERR_NONFINITE = -4
CLOTH_ERR_TIMEOUT = -5
CLOTH_ERR_BAD_MESH = -6
CLOTH_ERR_STATE = -7
CLOTH_FLAG_NO_GRAPH = 1
CLOTH_FLAG_ATOMIC_SPRINGS = 2
CLOTH_FLAG_EDGE_COLLISION = 4

_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NONFINITE", -5: "TIMEOUT",
          -6: "BAD_MESH", -7: "STATE"}

# Every symbol include/cloth.h declares (checked by the CPU test-suite).
EXPORTS = ("cloth_create", "cloth_set_mesh", "cloth_step", "cloth_read", "cloth_destroy",
           "cloth_set_state", "cloth_sync", "cloth_get_collision_stats", "cloth_last_error", "cloth_get_info", "cloth_get_grid",
           "cloth_query_candidates", "cloth_grid_build_static", "cloth_profile_substeps",
           "cloth_compute_normals",
           "cloth_batch_create", "cloth_batch_set_mesh", "cloth_batch_step", "cloth_batch_read",
           "cloth_batch_set_state", "cloth_batch_tune", "cloth_batch_set_tuning", "cloth_batch_get_tuning",
           "cloth_batch_sync", "cloth_batch_get_collision_stats", "cloth_batch_destroy",
           "cloth_rollout_create", "cloth_rollout_forward", "cloth_rollout_backward", "cloth_rollout_destroy")


class ClothError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"CLOTH_ERR_{_NAMES.get(code, code)} ({code}): {msg}")
        self.code = code


class ClothWind(C.Structure):
    _fields_ = [("amp", C.c_float), ("dir", C.c_float * 3), ("udir", C.c_float * 3), ("freq", C.c_float),
                ("kappa", C.c_float), ("phase", C.c_float)]


class ClothDesc(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("origin", C.c_float * 3), ("du", C.c_float * 3), ("dv", C.c_float * 3),
        ("total_mass", C.c_float),
        ("ks", C.c_float * 3), ("kd", C.c_float * 3),
        ("ks_spring", C.POINTER(C.c_float)), ("kd_spring", C.POINTER(C.c_float)),
        ("init_pos", C.POINTER(C.c_float)), ("init_vel", C.POINTER(C.c_float)),
        ("pinned", C.POINTER(C.c_uint8)),
        ("gravity", C.c_float * 3),
        ("dt", C.c_float), ("substeps", C.c_int32),
        ("contact_offset", C.c_float), ("mt_eps", C.c_float), ("mt_t_min", C.c_float),
        ("restitution", C.c_float),
        ("wind", ClothWind),
        ("flags", C.c_uint32),
        ("pin_velocity", C.c_float * 3),
    ]


class ClothInfo(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("n", C.c_int32), ("substeps", C.c_int32),
        ("substeps_done", C.c_int64), ("plane_stride", C.c_int64),
        ("pos_planes", C.c_void_p * 3), ("vel_planes", C.c_void_p * 3),
        ("ntris", C.c_int32), ("grid_dims", C.c_int32 * 3), ("grid_origin", C.c_float * 3),
        ("grid_h", C.c_float), ("grid_inv", C.c_float), ("grid_entries", C.c_int64),
        ("has_per_spring", C.c_int32), ("row_pitch", C.c_int32),
    ]


class ClothGridParams(C.Structure):
    _fields_ = [("h", C.c_float), ("inv", C.c_float), ("origin", C.c_float * 3), ("dims", C.c_int32 * 3),
                ("ncells", C.c_int64), ("nentries", C.c_int64)]


class ClothBatchTuning(C.Structure):
    _fields_ = [("rows_per_warp", C.c_int32), ("walk_ctas_per_sm", C.c_int32), ("us_per_substep", C.c_float),
                ("candidates", C.c_int32)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libcloth.so (built by paper_2507_11794_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2507_11794_gb300.build.build() "
                              "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        fp, ip, u8 = C.POINTER(C.c_float), C.POINTER(C.c_int32), C.POINTER(C.c_uint8)
        H = C.c_void_p
        L.cloth_create.argtypes = [C.POINTER(ClothDesc), C.c_void_p, C.POINTER(C.c_void_p)]
        L.cloth_set_mesh.argtypes = [H, fp, C.c_int32, ip, C.c_int32]
        L.cloth_step.argtypes = [H, C.c_int32]
        L.cloth_read.argtypes = [H, fp, fp]
        L.cloth_destroy.argtypes = [H]
        L.cloth_destroy.restype = None
        L.cloth_set_state.argtypes = [H, fp, fp]
        L.cloth_sync.argtypes = [H]
        L.cloth_get_collision_stats.argtypes = [H, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                                C.POINTER(C.c_int64)]
        L.cloth_last_error.argtypes = []
        L.cloth_last_error.restype = C.c_char_p
        L.cloth_get_info.argtypes = [H, C.POINTER(ClothInfo)]
        L.cloth_get_grid.argtypes = [H, ip, ip]
        L.cloth_query_candidates.argtypes = [H, fp, fp, C.c_int32, ip, ip, C.c_int32]
        L.cloth_grid_build_static.argtypes = [fp, C.c_int32, ip, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_int64, C.c_void_p, C.c_int64, C.POINTER(ClothGridParams)]
        L.cloth_batch_create.argtypes = [C.POINTER(ClothDesc), C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]
        L.cloth_batch_set_mesh.argtypes = [H, C.c_int32, fp, C.c_int32, ip, C.c_int32]
        L.cloth_batch_step.argtypes = [H, C.c_int32]
        L.cloth_batch_read.argtypes = [H, C.c_int32, fp, fp]
        L.cloth_batch_set_state.argtypes = [H, C.c_int32, fp, fp]
        L.cloth_batch_tune.argtypes = [H, C.c_int32, C.POINTER(ClothBatchTuning)]
        L.cloth_batch_set_tuning.argtypes = [H, C.c_int32, C.c_int32]
        L.cloth_batch_get_tuning.argtypes = [H, C.POINTER(ClothBatchTuning)]
        L.cloth_batch_sync.argtypes = [H]
        L.cloth_batch_get_collision_stats.argtypes = [H, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                                      C.POINTER(C.c_int64)]
        L.cloth_batch_destroy.argtypes = [H]
        L.cloth_batch_destroy.restype = None
        V = C.c_void_p
        L.cloth_rollout_create.argtypes = [H, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]
        L.cloth_rollout_forward.argtypes = [H, V, V, V, V, V]
        L.cloth_rollout_backward.argtypes = [H, V, V, V, V, V]
        L.cloth_rollout_destroy.argtypes = [H]
        L.cloth_rollout_destroy.restype = None
        for name in EXPORTS:
            f = getattr(L, name)
            if name not in ("cloth_destroy", "cloth_last_error", "cloth_batch_destroy", "cloth_rollout_destroy"):
                f.restype = C.c_int
        _lib = L
        return L


def check(rc: int):
    if rc < 0:
        raise ClothError(rc, lib().cloth_last_error().decode(errors="replace"))
    return rc


def _fp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_float))


def _ip(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int32))


def f32(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


# ---------------------------------------------------------------- C names

def cloth_create(desc: ClothDesc, stream: int = 0) -> int:
    h = C.c_void_p()
    check(lib().cloth_create(C.byref(desc), C.c_void_p(stream), C.byref(h)))
    return h.value


def cloth_set_mesh(h: int, verts, tris):
    v = None if verts is None else f32(verts, (-1, 3))
    t = None if tris is None else np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    nv = 0 if v is None else len(v)
    nt = 0 if t is None else len(t)
    check(lib().cloth_set_mesh(h, _fp(v), nv, _ip(t), nt))


def cloth_step(h: int, nsteps: int):
    check(lib().cloth_step(h, int(nsteps)))


def cloth_read(h: int, n: int, pos=True, vel=True, out_pos=None, out_vel=None):
    """Returns (pos, vel) as float32 (N,3) arrays (None for a part not read)."""
    p = (out_pos if out_pos is not None else np.empty((n, 3), np.float32)) if pos else None
    v = (out_vel if out_vel is not None else np.empty((n, 3), np.float32)) if vel else None
    check(lib().cloth_read(h, _fp(p), _fp(v)))
    return p, v


def cloth_set_state(h: int, pos=None, vel=None):
    check(lib().cloth_set_state(h, _fp(f32(pos)), _fp(f32(vel))))


def cloth_sync(h: int):
    check(lib().cloth_sync(h))


def cloth_get_collision_stats(h: int):
    """(listed, tested, hits): running collision totals since create."""
    v = [C.c_int64(0) for _ in range(3)]
    check(lib().cloth_get_collision_stats(h, *(C.byref(x) for x in v)))
    return tuple(int(x.value) for x in v)


def cloth_destroy(h: int):
    if h:
        lib().cloth_destroy(h)


def cloth_get_info(h: int) -> ClothInfo:
    info = ClothInfo()
    check(lib().cloth_get_info(h, C.byref(info)))
    return info


def cloth_compute_normals(h: int, d_normals_ptr: int):
    """Per-vertex normals into a device buffer of nx*ny*3 floats (async)."""
    check(lib().cloth_compute_normals(h, C.c_void_p(int(d_normals_ptr))))


def cloth_profile_substeps(h: int, nsub: int):
    """Mean device microseconds per launch of the walk and collision kernels
    over nsub substeps (the state advances)."""
    w, c = C.c_float(), C.c_float()
    check(lib().cloth_profile_substeps(h, int(nsub), C.byref(w), C.byref(c)))
    return float(w.value), float(c.value)


def cloth_get_grid(h: int):
    info = cloth_get_info(h)
    nc = int(info.grid_dims[0]) * int(info.grid_dims[1]) * int(info.grid_dims[2])
    cs = np.empty(nc + 1, np.int32)
    ids = np.empty(max(int(info.grid_entries), 1), np.int32)
    check(lib().cloth_get_grid(h, _ip(cs), _ip(ids)))
    return cs, ids[:int(info.grid_entries)]


def cloth_query_candidates(h: int, S, E, cap: int = 64):
    S = f32(S, (-1, 3))
    E = f32(E, (-1, 3))
    n = len(S)
    while True:
        counts = np.empty(n, np.int32)
        ids = np.empty((n, cap), np.int32)
        check(lib().cloth_query_candidates(h, _fp(S), _fp(E), n, _ip(counts), _ip(ids), cap))
        if n == 0 or counts.max() <= cap:
            return counts, ids
        cap = int(counts.max())


def cloth_grid_build_static(verts, tris, stream, d_tri_records, d_cell_start, cell_capacity, d_tri_ids,
                            entry_capacity):
    """Allocation-free grid build into caller device buffers (raw device
    addresses as ints).  Returns (status, ClothGridParams); does not raise, so
    callers can size buffers from a CLOTH_ERR_INVALID_ARG answer."""
    v = f32(verts, (-1, 3))
    t = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    prm = ClothGridParams()
    rc = lib().cloth_grid_build_static(_fp(v), len(v), _ip(t), len(t), C.c_void_p(stream),
                                       C.c_void_p(d_tri_records), C.c_void_p(d_cell_start), int(cell_capacity),
                                       C.c_void_p(d_tri_ids), int(entry_capacity), C.byref(prm))
    return rc, prm


# ---------------------------------------------------------------- batches

def cloth_batch_create(descs, stream: int = 0) -> int:
    arr = (ClothDesc * len(descs))(*descs)
    h = C.c_void_p()
    check(lib().cloth_batch_create(arr, len(descs), C.c_void_p(stream), C.byref(h)))
    return h.value


def cloth_batch_set_mesh(b: int, index: int, verts, tris):
    v = None if verts is None else f32(verts, (-1, 3))
    t = None if tris is None else np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    check(lib().cloth_batch_set_mesh(b, int(index), _fp(v), 0 if v is None else len(v), _ip(t),
                                     0 if t is None else len(t)))


def cloth_batch_step(b: int, nsteps: int):
    check(lib().cloth_batch_step(b, int(nsteps)))


def cloth_batch_read(b: int, index: int, n: int, pos=True, vel=True):
    p = np.empty((n, 3), np.float32) if pos else None
    v = np.empty((n, 3), np.float32) if vel else None
    check(lib().cloth_batch_read(b, int(index), _fp(p), _fp(v)))
    return p, v


def cloth_batch_set_state(b: int, index: int, pos=None, vel=None):
    check(lib().cloth_batch_set_state(b, int(index), _fp(f32(pos)), _fp(f32(vel))))


def cloth_batch_tune(b: int, trial_substeps: int = 20) -> ClothBatchTuning:
    t = ClothBatchTuning()
    check(lib().cloth_batch_tune(b, int(trial_substeps), C.byref(t)))
    return t


def cloth_batch_set_tuning(b: int, rows_per_warp: int, walk_ctas_per_sm: int):
    check(lib().cloth_batch_set_tuning(b, int(rows_per_warp), int(walk_ctas_per_sm)))


def cloth_batch_get_tuning(b: int) -> ClothBatchTuning:
    t = ClothBatchTuning()
    check(lib().cloth_batch_get_tuning(b, C.byref(t)))
    return t


def cloth_batch_sync(b: int):
    check(lib().cloth_batch_sync(b))


def cloth_batch_get_collision_stats(b: int):
    """(listed, tested, hits): running collision totals of the batch."""
    v = [C.c_int64(0) for _ in range(3)]
    check(lib().cloth_batch_get_collision_stats(b, *(C.byref(x) for x in v)))
    return tuple(int(x.value) for x in v)


def cloth_batch_destroy(b: int):
    if b:
        lib().cloth_batch_destroy(b)


# ---------------------------------------------------------------- rollouts

def cloth_rollout_create(h: int, nsteps: int, checkpoint_every: int) -> int:
    r = C.c_void_p()
    check(lib().cloth_rollout_create(h, int(nsteps), int(checkpoint_every), C.byref(r)))
    return r.value


def cloth_rollout_forward(r: int, d_ks: int, d_kd: int, d_v0: int, d_pos: int, d_vel: int):
    """Device addresses (ints, 0 = NULL)."""
    check(lib().cloth_rollout_forward(r, d_ks or None, d_kd or None, d_v0 or None, d_pos or None, d_vel or None))


def cloth_rollout_backward(r: int, d_gpos: int, d_gvel: int, d_gks: int, d_gkd: int, d_gv0: int):
    check(lib().cloth_rollout_backward(r, d_gpos or None, d_gvel or None, d_gks or None, d_gkd or None,
                                       d_gv0 or None))


def cloth_rollout_destroy(r: int):
    if r:
        lib().cloth_rollout_destroy(r)
