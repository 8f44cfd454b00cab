"""GB300-native mass-spring cloth stepping (arXiv 2507.11794's hot path).

The compute lives in libcloth.so (hand-written CUDA for sm_103a, C ABI in
include/cloth.h); this package is its thin Python face:

* ``capi``  -- ctypes binding with the C names (cloth_create, cloth_set_mesh,
               cloth_step, cloth_read, cloth_destroy, ...);
* ``Cloth`` -- a small owner object over one handle, built from a problem
               description (any object with the ClothDesc fields, e.g. a
               ``cloth_scenes.Scene``);
* ``rollout`` -- differentiable rollouts (torch.autograd.Function over the
               library's reverse pass);
* ``build`` -- the in-tree nvcc build.

PyTorch, when present, only supplies the CUDA stream (the current stream of
the current device).  There is no CPU fallback: without the library or a GPU
every call raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi
from .capi import ClothError

__all__ = ["Cloth", "ClothBatch", "ClothError", "capi", "make_desc", "current_stream"]


def current_stream() -> int:
    """cudaStream_t of torch's current stream (0 = legacy default stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def make_desc(p, keep: list, flags: int = 0) -> capi.ClothDesc:
    """Fill a ClothDesc from an object with the problem fields; arrays are
    converted to contiguous numpy buffers appended to ``keep`` (they must
    outlive the create call)."""
    d = capi.ClothDesc()
    d.nx, d.ny = int(p.nx), int(p.ny)
    for k in range(3):
        d.origin[k], d.du[k], d.dv[k] = p.origin[k], p.du[k], p.dv[k]
        d.ks[k], d.kd[k], d.gravity[k] = p.ks[k], p.kd[k], p.gravity[k]
        d.wind.dir[k], d.wind.udir[k] = p.wind.dir[k], p.wind.udir[k]
    d.total_mass = p.total_mass
    d.dt, d.substeps = p.dt, int(p.substeps)
    d.contact_offset, d.mt_eps = p.contact_offset, p.mt_eps
    d.mt_t_min, d.restitution = p.mt_t_min, p.restitution
    d.wind.amp, d.wind.freq, d.wind.kappa, d.wind.phase = p.wind.amp, p.wind.freq, p.wind.kappa, p.wind.phase
    d.flags = int(flags)
    for k in range(3):
        d.pin_velocity[k] = float(getattr(p, "pin_velocity", (0.0, 0.0, 0.0))[k])
    N = d.nx * d.ny

    def fbuf(a, n):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
        if a.size != n:
            raise ValueError(f"array of {a.size} floats, expected {n}")
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_float))

    d.init_pos = fbuf(getattr(p, "init_pos", None), 3 * N)
    d.init_vel = fbuf(getattr(p, "init_vel", None), 3 * N)
    S = None
    if getattr(p, "ks_spring", None) is not None or getattr(p, "kd_spring", None) is not None:
        a = p.ks_spring if p.ks_spring is not None else p.kd_spring
        S = int(np.asarray(a).size)
    d.ks_spring = fbuf(getattr(p, "ks_spring", None), S)
    d.kd_spring = fbuf(getattr(p, "kd_spring", None), S)
    pin = getattr(p, "pinned", None)
    if pin is not None:
        pin = np.ascontiguousarray(pin, dtype=np.uint8).reshape(-1)
        if pin.size != N:
            raise ValueError("pinned must have N entries")
        keep.append(pin)
        d.pinned = pin.ctypes.data_as(C.POINTER(C.c_uint8))
    return d


class Cloth:
    """One cloth on the GPU (owner of a ClothHandle)."""

    def __init__(self, problem, stream: int | None = None, flags: int = 0, mesh: bool = True):
        keep: list = []
        desc = make_desc(problem, keep, flags)
        self.n = desc.nx * desc.ny
        self.nx, self.ny = desc.nx, desc.ny
        self.substeps = desc.substeps
        self.h = capi.cloth_create(desc, current_stream() if stream is None else stream)
        if mesh and getattr(problem, "mesh_tris", None) is not None and len(problem.mesh_tris):
            self.set_mesh(problem.mesh_verts, problem.mesh_tris)

    def set_mesh(self, verts, tris):
        capi.cloth_set_mesh(self.h, verts, tris)

    def step(self, nsteps: int = 1):
        capi.cloth_step(self.h, nsteps)

    def read(self, pos=True, vel=True, out_pos=None, out_vel=None):
        return capi.cloth_read(self.h, self.n, pos, vel, out_pos, out_vel)

    def set_state(self, pos=None, vel=None):
        capi.cloth_set_state(self.h, pos, vel)

    def sync(self):
        capi.cloth_sync(self.h)

    def info(self):
        return capi.cloth_get_info(self.h)

    def collision_stats(self):
        """(listed, tested, hits) summed over all substeps since create."""
        return capi.cloth_get_collision_stats(self.h)

    def normals(self, out=None):
        """Per-vertex normals of the current state as a (N, 3) float32 CUDA
        tensor (``out`` if given)."""
        import torch
        if out is None:
            out = torch.empty((self.n, 3), dtype=torch.float32, device="cuda")
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.numel() == 3 * self.n
        capi.cloth_compute_normals(self.h, out.data_ptr())
        return out

    def profile_substeps(self, nsub: int):
        """(walk_us, collide_us): mean device time per launch of each kernel."""
        return capi.cloth_profile_substeps(self.h, nsub)

    def grid(self):
        return capi.cloth_get_grid(self.h)

    def query_candidates(self, S, E, cap: int = 64):
        return capi.cloth_query_candidates(self.h, S, E, cap)

    def close(self):
        if getattr(self, "h", None):
            capi.cloth_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class ClothBatch:
    """Many independent cloths stepped together (owner of a ClothBatch)."""

    def __init__(self, problems, stream: int | None = None, flags: int = 0, mesh: bool = True):
        keep: list = []
        descs = [make_desc(p, keep, flags) for p in problems]
        self.sizes = [d.nx * d.ny for d in descs]
        self.h = capi.cloth_batch_create(descs, current_stream() if stream is None else stream)
        if mesh:
            for i, p in enumerate(problems):
                if getattr(p, "mesh_tris", None) is not None and len(p.mesh_tris):
                    capi.cloth_batch_set_mesh(self.h, i, p.mesh_verts, p.mesh_tris)

    def __len__(self):
        return len(self.sizes)

    def step(self, nsteps: int = 1):
        capi.cloth_batch_step(self.h, nsteps)

    def read(self, index: int, pos=True, vel=True):
        return capi.cloth_batch_read(self.h, index, self.sizes[index], pos, vel)

    def set_state(self, index: int, pos=None, vel=None):
        capi.cloth_batch_set_state(self.h, index, pos, vel)

    def tune(self, trial_substeps: int = 20):
        return capi.cloth_batch_tune(self.h, trial_substeps)

    def set_tuning(self, rows_per_warp: int, walk_ctas_per_sm: int):
        capi.cloth_batch_set_tuning(self.h, rows_per_warp, walk_ctas_per_sm)

    def tuning(self):
        return capi.cloth_batch_get_tuning(self.h)

    def collision_stats(self):
        """(listed, tested, hits) of the whole batch since create."""
        return capi.cloth_batch_get_collision_stats(self.h)

    def sync(self):
        capi.cloth_batch_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            capi.cloth_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
