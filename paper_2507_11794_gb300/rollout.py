"""Differentiable rollouts: torch.autograd.Function over the C ABI's
cloth_rollout_* (hand-written reverse pass in libcloth.so, step checkpoints).

    cl = Cloth(problem)                      # any cloth; its state is x0
    ro = Rollout(cl, nsteps=256, checkpoint_every=16)
    pos, vel = ro(ks, kd, v0)                # CUDA float32 tensors
    loss = ((pos - target) ** 2).sum(1).mean()
    loss.backward()                          # ks.grad, kd.grad, v0.grad

ks, kd: (S,) per-spring constants in canonical order; v0: (N, 3).  Torch
only supplies device memory and the stream; the forward and backward passes
run in the library's kernels.
"""
from __future__ import annotations

import torch

from . import capi


class _RolloutFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ks, kd, v0, ro):
        n = ro.cloth.n
        pos = torch.empty((n, 3), dtype=torch.float32, device=ks.device)
        vel = torch.empty((n, 3), dtype=torch.float32, device=ks.device)
        capi.cloth_rollout_forward(ro.r, ks.data_ptr(), kd.data_ptr(), v0.data_ptr(), pos.data_ptr(),
                                   vel.data_ptr())
        ctx.ro = ro
        ctx.shapes = (ks.shape, kd.shape, v0.shape)
        return pos, vel

    @staticmethod
    def backward(ctx, gpos, gvel):
        ro = ctx.ro
        dev = gpos.device if gpos is not None else gvel.device
        s_ks, s_kd, s_v0 = ctx.shapes
        gks = torch.empty(s_ks, dtype=torch.float32, device=dev)
        gkd = torch.empty(s_kd, dtype=torch.float32, device=dev)
        gv0 = torch.empty(s_v0, dtype=torch.float32, device=dev)
        gp = gpos.contiguous() if gpos is not None else torch.zeros((ro.cloth.n, 3), device=dev)
        gv = gvel.contiguous() if gvel is not None else None
        capi.cloth_rollout_backward(ro.r, gp.data_ptr(), gv.data_ptr() if gv is not None else 0, gks.data_ptr(),
                                    gkd.data_ptr(), gv0.data_ptr())
        return gks, gkd, gv0, None


class Rollout:
    """nsteps steps of a Cloth from its current state, differentiable in the
    per-spring constants and the initial velocities."""

    def __init__(self, cloth, nsteps: int, checkpoint_every: int = 16):
        self.cloth = cloth
        self.r = capi.cloth_rollout_create(cloth.h, nsteps, checkpoint_every)

    def __call__(self, ks: torch.Tensor, kd: torch.Tensor, v0: torch.Tensor):
        for t in (ks, kd, v0):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("ks, kd, v0 must be contiguous CUDA float32 tensors")
        return _RolloutFn.apply(ks, kd, v0, self)

    def close(self):
        if getattr(self, "r", None):
            capi.cloth_rollout_destroy(self.r)
            self.r = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
