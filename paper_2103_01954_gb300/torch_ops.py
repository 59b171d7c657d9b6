"""PyTorch-facing wrapper around the C ABI: tensors supply device pointers and the
current CUDA stream; every computation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import binding as B

_DT = {torch.float32: B.MVP_F32, torch.bfloat16: B.MVP_BF16, torch.float16: B.MVP_F16}


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t: torch.Tensor, name: str, dtype=None, shape_tail=None):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if shape_tail is not None and tuple(t.shape[-len(shape_tail):]) != tuple(shape_tail):
        raise ValueError(f"{name} has shape {tuple(t.shape)}")


def prims_struct(t, q, s, payload) -> B.mvp_prims:
    """mvp_prims from t [N,3], q [N,4], s [N,3] float32 and payload [N,M,M,M,4]."""
    _need(t, "t", torch.float32, (3,))
    _need(q, "q", torch.float32, (4,))
    _need(s, "s", torch.float32, (3,))
    _need(payload, "payload")
    if payload.dtype not in _DT:
        raise ValueError(f"payload dtype {payload.dtype} unsupported")
    n = t.shape[0]
    if payload.dim() != 5 or payload.shape[0] != n or payload.shape[4] != 4:
        raise ValueError(f"payload shape {tuple(payload.shape)}")
    M = payload.shape[1]
    return B.mvp_prims(n=n, M=M, dtype=_DT[payload.dtype], reserved=0, t=_ptr(t), q=_ptr(q), s=_ptr(s),
                       payload=_ptr(payload))


def rays_struct(o, d, t_near, t_far, dt, eps_early=0.0, bg=(0.0, 0.0, 0.0), width=0, height=0,
                sequential=False, literal_composite=False) -> B.mvp_rays:
    """mvp_rays; sequential=True blends a ray's saturating sample in BVH order;
    literal_composite=True composites A I + (1 - A) B."""
    _need(o, "o", torch.float32, (3,))
    _need(d, "d", torch.float32, (3,))
    r = B.mvp_rays(n=o.shape[0], o=_ptr(o), d=_ptr(d), t_near=t_near, t_far=t_far, dt=dt, eps_early=eps_early,
                   width=width, height=height,
                   flags=(B.MVP_BLEND_SEQUENTIAL if sequential else 0) |
                   (B.MVP_COMPOSITE_LITERAL if literal_composite else 0))
    r.bg[0], r.bg[1], r.bg[2] = bg
    return r


class Context:
    """An mvp_ctx bound to one CUDA device."""

    def __init__(self, device: int | None = None):
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        B.check(B.lib().mvp_ctx_create(self.device, ctypes.byref(h)), "mvp_ctx_create")
        self.handle = h

    def sync(self):
        B.check(B.lib().mvp_ctx_sync(self.handle, _stream()), "mvp_ctx_sync")

    def set_tile_schedule(self, enable: bool):
        """Heaviest tiles of the last frame first (default), or the plain tile order."""
        B.check(B.lib().mvp_ctx_set_tile_schedule(self.handle, 1 if enable else 0), "mvp_ctx_set_tile_schedule")

    def set_bwd_group_bytes(self, nbytes: int):
        """Adjoint primitive-group size in bytes (0: a third of L2, the default; < 0: never group)."""
        B.check(B.lib().mvp_ctx_set_bwd_group_bytes(self.handle, int(nbytes)), "mvp_ctx_set_bwd_group_bytes")

    def close(self):
        if self.handle:
            B.lib().mvp_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BVH:
    """An mvp_bvh handle (library-owned device buffers, reused across frames)."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        h = ctypes.c_void_p()
        B.check(B.lib().mvp_bvh_create(ctx.handle, ctypes.byref(h)), "mvp_bvh_create")
        self.handle = h

    def build(self, prims: B.mvp_prims):
        B.check(B.lib().mvp_build_bvh(self.ctx.handle, ctypes.byref(prims), self.handle, _stream()), "mvp_build_bvh")

    @property
    def size(self) -> int:
        return B.lib().mvp_bvh_size(self.handle)

    def export(self):
        n = self.size
        dev = torch.device("cuda", self.ctx.device)
        keys = torch.empty(max(n, 0), dtype=torch.int64, device=dev)
        children = torch.empty((max(n - 1, 0), 2), dtype=torch.int32, device=dev)
        bounds = torch.empty((max(2 * n - 1, 0), 6), dtype=torch.float32, device=dev)
        scene = torch.empty(6, dtype=torch.float32, device=dev)
        B.check(B.lib().mvp_bvh_export(self.ctx.handle, self.handle, _ptr(keys), _ptr(children), _ptr(bounds),
                                       _ptr(scene), _stream()), "mvp_bvh_export")
        return keys, children, bounds, scene

    def close(self):
        if self.handle:
            B.lib().mvp_bvh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def saved_bytes(n_rays: int) -> int:
    return int(B.lib().mvp_saved_bytes(n_rays))


def raymarch_fwd(ctx: Context, prims, bvh: BVH, rays, out=None, saved=None, want_saved=False):
    dev = torch.device("cuda", ctx.device)
    if out is None:
        out = torch.empty((rays.n, 4), dtype=torch.float32, device=dev)
    if want_saved and saved is None:
        saved = torch.empty(saved_bytes(rays.n), dtype=torch.uint8, device=dev)
    B.check(B.lib().mvp_raymarch_fwd(ctx.handle, ctypes.byref(prims), bvh.handle, ctypes.byref(rays), _ptr(out),
                                     _ptr(saved), _stream()), "mvp_raymarch_fwd")
    return out, saved


def raymarch_count(ctx: Context, prims, bvh: BVH, rays):
    n_eval = torch.empty(rays.n, dtype=torch.int32, device=torch.device("cuda", ctx.device))
    B.check(B.lib().mvp_raymarch_count(ctx.handle, ctypes.byref(prims), bvh.handle, ctypes.byref(rays),
                                       _ptr(n_eval), _stream()), "mvp_raymarch_count")
    return n_eval


def raymarch_bwd(ctx: Context, prims, bvh: BVH, rays, saved, grad_rgba, g_payload=None, g_t=None, g_q=None,
                 g_s=None):
    _need(grad_rgba, "grad_rgba", torch.float32, (4,))
    B.check(B.lib().mvp_raymarch_bwd(ctx.handle, ctypes.byref(prims), bvh.handle, ctypes.byref(rays),
                                     _ptr(saved), _ptr(grad_rgba), _ptr(g_payload), _ptr(g_t), _ptr(g_q),
                                     _ptr(g_s), _stream()), "mvp_raymarch_bwd")


def hitlists(ctx: Context, prims, bvh: BVH, rays, cap: int | None = None):
    """CSR hit lists: (offs [R+1] int64, ids int32, tin, tout float32), synchronising."""
    dev = torch.device("cuda", ctx.device)
    offs = torch.empty(rays.n + 1, dtype=torch.int64, device=dev)
    n_hits = ctypes.c_int64(0)
    st = B.lib().mvp_hitlists(ctx.handle, ctypes.byref(prims), bvh.handle, ctypes.byref(rays), _ptr(offs), None,
                              None, None, 0, ctypes.byref(n_hits), _stream())
    if st not in (B.MVP_OK, B.MVP_ERR_CAPACITY):
        B.check(st, "mvp_hitlists(count)")
    cap = int(n_hits.value) if cap is None else cap
    ids = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    tin = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
    tout = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
    B.check(B.lib().mvp_hitlists(ctx.handle, ctypes.byref(prims), bvh.handle, ctypes.byref(rays), _ptr(offs),
                                 _ptr(ids), _ptr(tin), _ptr(tout), cap, ctypes.byref(n_hits), _stream()),
            "mvp_hitlists")
    H = int(n_hits.value)
    return offs, ids[:H], tin[:H], tout[:H]


def pack_payload(ctx: Context, payload_f32: torch.Tensor, dtype: torch.dtype) -> torch.Tensor:
    _need(payload_f32, "payload", torch.float32)
    out = torch.empty(payload_f32.shape, dtype=dtype, device=payload_f32.device)
    B.check(B.lib().mvp_pack_payload(ctx.handle, _ptr(payload_f32), _ptr(out), payload_f32.numel(), _DT[dtype],
                                     _stream()), "mvp_pack_payload")
    return out


def fade_payload(ctx: Context, payload_f32: torch.Tensor, dtype: torch.dtype = torch.float32, alpha: float = 8.0,
                 beta: int = 8, out: torch.Tensor | None = None) -> torch.Tensor:
    """mvp_fade_payload: opacity multiplied by the fade window, converted to `dtype`.
    payload_f32 is [n, M, M, M, 4]; out may be payload_f32 itself when dtype is FP32."""
    _need(payload_f32, "payload", torch.float32)
    n, M = payload_f32.shape[0], payload_f32.shape[1]
    if out is None:
        out = torch.empty(payload_f32.shape, dtype=dtype, device=payload_f32.device)
    B.check(B.lib().mvp_fade_payload(ctx.handle, _ptr(payload_f32), _ptr(out), n, M, _DT[dtype], float(alpha),
                                     int(beta), _stream()), "mvp_fade_payload")
    return out


def assemble_payload(ctx: Context, rgb: torch.Tensor, opacity: torch.Tensor, dtype: torch.dtype = torch.bfloat16,
                     alpha: float = 8.0, beta: int = 8, out: torch.Tensor | None = None) -> torch.Tensor:
    """mvp_assemble_payload: a view's payload [n, M, M, M, 4] in `dtype` from its
    view-dependent colour rgb [n, M, M, M, 3] and the shared opacity [n, M, M, M]
    (faded with alpha, beta; alpha = 0: no fade)."""
    _need(rgb, "rgb", torch.float32, (3,))
    _need(opacity, "opacity", torch.float32)
    n, M = rgb.shape[0], rgb.shape[1]
    if tuple(opacity.shape) != tuple(rgb.shape[:-1]):
        raise ValueError("opacity must be rgb's shape without the channel axis")
    if out is None:
        out = torch.empty((n, M, M, M, 4), dtype=dtype, device=rgb.device)
    B.check(B.lib().mvp_assemble_payload(ctx.handle, _ptr(rgb), _ptr(opacity), _ptr(out), n, M, _DT[dtype],
                                         float(alpha), int(beta), _stream()), "mvp_assemble_payload")
    return out


def axis_angle_to_quat(ctx: Context, r: torch.Tensor) -> torch.Tensor:
    _need(r, "r", torch.float32, (3,))
    q = torch.empty((r.shape[0], 4), dtype=torch.float32, device=r.device)
    B.check(B.lib().mvp_axis_angle_to_quat(ctx.handle, _ptr(r), r.shape[0], _ptr(q), _stream()),
            "mvp_axis_angle_to_quat")
    return q


def axis_angle_backward(ctx: Context, r: torch.Tensor, g_q: torch.Tensor, g_r: torch.Tensor | None = None):
    """g_r += (dq/dr)^T g_q; returns g_r."""
    _need(r, "r", torch.float32, (3,))
    _need(g_q, "g_q", torch.float32, (4,))
    if g_r is None:
        g_r = torch.zeros_like(r)
    B.check(B.lib().mvp_axis_angle_backward(ctx.handle, _ptr(r), _ptr(g_q), r.shape[0], _ptr(g_r), _stream()),
            "mvp_axis_angle_backward")
    return g_r


def volume_prior(ctx: Context, s: torch.Tensor, lam: float = 0.01, g_s: torch.Tensor | None = None):
    """Returns (loss tensor [1], g_s) with g_s += dL_vol/ds (g_s None: no gradient)."""
    _need(s, "s", torch.float32, (3,))
    loss = torch.zeros(1, dtype=torch.float32, device=s.device)
    B.check(B.lib().mvp_volume_prior(ctx.handle, _ptr(s), s.shape[0], float(lam), _ptr(loss), _ptr(g_s),
                                     _stream()), "mvp_volume_prior")
    return loss, g_s


def camera_rays(ctx: Context, c2w, focal: float, width: int, height: int, out=None):
    """mvp_camera_rays: (o, d) [width * height, 3] of a pinhole camera; out = (o, d)
    writes into given tensors."""
    dev = torch.device("cuda", ctx.device)
    if out is not None:
        o, d = out
        _need(o, "o", torch.float32, (3,))
        _need(d, "d", torch.float32, (3,))
    else:
        o = torch.empty((width * height, 3), dtype=torch.float32, device=dev)
        d = torch.empty((width * height, 3), dtype=torch.float32, device=dev)
    m = (ctypes.c_float * 12)(*[float(v) for v in list(c2w.reshape(-1))])
    B.check(B.lib().mvp_camera_rays(ctx.handle, m, float(focal), width, height, _ptr(o), _ptr(d), _stream()),
            "mvp_camera_rays")
    return o, d


def allreduce_gradients(grads, group=None):
    """The data-parallel backward's one exchange: ranks that marched disjoint sets of
    rays (cameras, image rows) over the same primitives hold partial gradients whose
    sum is the gradient of the whole batch (the loss is a sum over rays). Sums the
    given tensors over the process group in place, as one flat collective (NCCL for
    device tensors, gloo for host tensors). A no-op without an initialised group."""
    import torch.distributed as dist

    grads = [g for g in grads if g is not None]
    if not grads or not dist.is_available() or not dist.is_initialized():
        return grads
    flat = torch.cat([g.reshape(-1) for g in grads])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for g in grads:
        n = g.numel()
        g.copy_(flat[off:off + n].view_as(g))
        off += n
    return grads


class MVPRender(torch.autograd.Function):
    """Differentiable render: (t, q, s, payload) -> rgba [R, 4].

    Forward rebuilds the BVH (the per-frame rebuild of Sec. 3.2.1) and marches with
    saved per-ray state; backward replays the march (mvp_raymarch_bwd)."""

    @staticmethod
    def forward(fctx, t, q, s, payload, o, d, params: dict, ctx: Context, bvh: BVH):
        prims = prims_struct(t, q, s, payload)
        rays = rays_struct(o, d, **params)
        bvh.build(prims)
        out, saved = raymarch_fwd(ctx, prims, bvh, rays, want_saved=True)
        fctx.save_for_backward(t, q, s, payload, o, d, saved)
        fctx.params, fctx.mctx, fctx.bvh = params, ctx, bvh
        return out

    @staticmethod
    def backward(fctx, grad_out):
        t, q, s, payload, o, d, saved = fctx.saved_tensors
        prims = prims_struct(t, q, s, payload)
        rays = rays_struct(o, d, **fctx.params)
        need_p, need_pose = fctx.needs_input_grad[3], any(fctx.needs_input_grad[0:3])
        g_payload = torch.zeros(payload.shape, dtype=torch.float32, device=payload.device) if need_p else None
        g_t = torch.zeros_like(t) if need_pose else None
        g_q = torch.zeros_like(q) if need_pose else None
        g_s = torch.zeros_like(s) if need_pose else None
        # the handle may hold another frame's hierarchy by now; rebuilding is exact
        fctx.bvh.build(prims)
        raymarch_bwd(fctx.mctx, prims, fctx.bvh, rays, saved, grad_out.contiguous().float(), g_payload, g_t, g_q,
                     g_s)
        if g_payload is not None and payload.dtype != torch.float32:
            g_payload = g_payload.to(payload.dtype)
        return g_t, g_q, g_s, g_payload, None, None, None, None, None


def render(t, q, s, payload, o, d, params: dict, ctx: Context, bvh: BVH):
    return MVPRender.apply(t, q, s, payload, o, d, params, ctx, bvh)


class Server:
    """mvp_server: continuous batching of render requests over resident avatars."""

    def __init__(self, ctx: Context, hbm_budget: int, max_slots: int = 64, arena_bytes: int = 0):
        self.ctx = ctx
        h = ctypes.c_void_p()
        B.check(B.lib().mvp_serve_create(ctx.handle, int(hbm_budget), int(max_slots), int(arena_bytes),
                                         ctypes.byref(h)), "mvp_serve_create")
        self.handle = h
        self._keep = []  # avatar tensors must outlive the server

    def register(self, t, q, s, payload) -> int:
        prims = prims_struct(t, q, s, payload)
        aid = ctypes.c_int32(-1)
        B.check(B.lib().mvp_serve_register_avatar(self.handle, ctypes.byref(prims), ctypes.byref(aid)),
                "mvp_serve_register_avatar")
        self._keep.append((t, q, s, payload))
        return aid.value

    @staticmethod
    def request(avatar: int, c2w, focal: float, width: int, height: int, t_near: float, t_far: float, dt: float,
                eps_early: float = 0.0, bg=(0.0, 0.0, 0.0), c2w_right=None, payload=None) -> B.mvp_request:
        """A request; with c2w_right, a stereo pair whose image is [2][height][width][4];
        with payload (a device tensor in the avatar's layout and dtype), the request
        renders that payload instead of the avatar's (the caller keeps it alive until
        the request completes)."""
        r = B.mvp_request(avatar=avatar, width=width, height=height, focal=focal, t_near=t_near, t_far=t_far, dt=dt,
                          eps_early=eps_early, views=1 if c2w_right is None else 2,
                          payload=None if payload is None else payload.data_ptr())
        for i, v in enumerate([float(x) for x in list(c2w.reshape(-1))]):
            r.c2w[i] = v
        if c2w_right is not None:
            for i, v in enumerate([float(x) for x in list(c2w_right.reshape(-1))]):
                r.c2w_right[i] = v
        r.bg[0], r.bg[1], r.bg[2] = bg
        return r

    def submit_raw(self, req: B.mvp_request) -> int:
        """Returns the ticket; raises on refusal."""
        tk = ctypes.c_uint64(0)
        B.check(B.lib().mvp_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(tk)), "mvp_serve_submit")
        return tk.value

    def poll(self, ticket: int, out=None):
        """(status, latency_ms); status is MVP_OK or MVP_NOT_READY."""
        lat = ctypes.c_double(0.0)
        st = B.lib().mvp_serve_poll(self.handle, ticket, _ptr(out), ctypes.byref(lat))
        if st < 0:
            B.check(st, "mvp_serve_poll")
        return st, lat.value

    def wait(self, ticket: int, timeout_ms: float, out=None):
        lat = ctypes.c_double(0.0)
        st = B.lib().mvp_serve_wait(self.handle, ticket, float(timeout_ms), _ptr(out), ctypes.byref(lat))
        return st, lat.value

    def cancel(self, ticket: int) -> None:
        """Withdraw a request (queued: dropped; running: finishes, then freed)."""
        B.check(B.lib().mvp_serve_cancel(self.handle, ctypes.c_uint64(ticket)), "mvp_serve_cancel")

    def stats(self) -> dict:
        info = B.mvp_serve_info()
        B.check(B.lib().mvp_serve_stats(self.handle, ctypes.byref(info)), "mvp_serve_stats")
        return {k: getattr(info, k) for k, _ in B.mvp_serve_info._fields_}

    def close(self):
        if self.handle:
            B.lib().mvp_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
