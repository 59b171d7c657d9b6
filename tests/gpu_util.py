"""Helpers for GPU tests: move seeded scenes/rays to the device and call the C ABI
through the binding (paper_2103_01954_gb300.torch_ops)."""
from __future__ import annotations

import numpy as np
import torch

from paper_2103_01954_gb300 import torch_ops as T

DEV = torch.device("cuda", 0)


class Dev:
    """A scene + rays on the device with their ABI structs."""

    def __init__(self, scene, rays, payload_dtype=torch.float32, ctx=None):
        self.scene, self.rays = scene, rays
        self.t = torch.from_numpy(np.ascontiguousarray(scene.t)).to(DEV)
        self.q = torch.from_numpy(np.ascontiguousarray(scene.q)).to(DEV)
        self.s = torch.from_numpy(np.ascontiguousarray(scene.s)).to(DEV)
        p32 = torch.from_numpy(np.ascontiguousarray(scene.payload)).to(DEV)
        self.ctx = ctx or T.Context(0)
        self.payload = p32 if payload_dtype == torch.float32 else T.pack_payload(self.ctx, p32, payload_dtype)
        self.o = torch.from_numpy(np.ascontiguousarray(rays.o)).to(DEV)
        self.d = torch.from_numpy(np.ascontiguousarray(rays.d)).to(DEV)
        self.prims = T.prims_struct(self.t, self.q, self.s, self.payload)
        self.params = dict(t_near=rays.t_near, t_far=rays.t_far, dt=rays.dt, eps_early=rays.eps_early,
                           bg=tuple(rays.bg), width=rays.width, height=rays.height)
        self.rs = T.rays_struct(self.o, self.d, **self.params)
        self.bvh = T.BVH(self.ctx)

    def build(self):
        self.bvh.build(self.prims)
        return self

    def render(self, want_saved=False):
        out, saved = T.raymarch_fwd(self.ctx, self.prims, self.bvh, self.rs, want_saved=want_saved)
        self.ctx.sync()
        return out, saved

    def hitlists(self):
        return T.hitlists(self.ctx, self.prims, self.bvh, self.rs)

    def count(self):
        n = T.raymarch_count(self.ctx, self.prims, self.bvh, self.rs)
        self.ctx.sync()
        return n


def image_parity(gpu: np.ndarray, ref: np.ndarray, near_face: np.ndarray | None = None):
    """Statistics of |gpu - ref| per pixel channel."""
    err = np.abs(gpu.astype(np.float64) - ref)
    return {"max": float(err.max()) if err.size else 0.0,
            "frac_2e-4": float((err <= 2e-4).mean()) if err.size else 1.0,
            "p999": float(np.quantile(err, 0.999)) if err.size else 0.0}
