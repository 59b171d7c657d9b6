"""The allocation-free render entry point (mvp_raymarch_fwd_static).

It exists for callers that cannot allocate device memory (a plug-in inside an
application that owns the device allocator, a frame loop that must not stall on
cudaMalloc/cudaFree). It keeps its BVH in a fixed device array inside the library,
so it must give the same image as the allocating path (mvp_build_bvh +
mvp_raymarch_fwd) on every call, including a call that follows another scene, and it
must not change the device's free memory. This file is collected last on purpose.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import synthetic
from helpers import rays_from

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from gpu_util import DEV, Dev  # noqa: E402
from paper_2103_01954_gb300 import binding as B  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _static_render(dv, out, status):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = B.lib().mvp_raymarch_fwd_static(ctypes.byref(dv.prims), ctypes.byref(dv.rs),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(status.data_ptr()), stream)
    B.check(st, "mvp_raymarch_fwd_static")
    torch.cuda.synchronize()


def _scenes():
    """Scenes in the order the shared array sees them: a 4096-primitive FP32 frame, the
    same again, a smaller 8^3 one, a BF16 one with 32^3 payloads, a 12000-primitive one
    (more than one block sorts: the multi-pass radix sort inside the array), an empty
    one with a coloured background, and the first again."""
    a = Dev(*synthetic.make_config("small_4096x16^3_83x128", 0)[:2]).build()
    b = Dev(*synthetic.make_config("small_512x8^3_96x128", 1)[:2], ctx=a.ctx).build()
    sc, rays, _ = synthetic.make_config("diff_small_64x8^3_2x48x40", 2)
    big = synthetic.make_scene(96, 32, 3, layout="shell", s_range=(0.2, 0.4), empty_frac=0.6)
    c = Dev(big, rays, payload_dtype=torch.bfloat16, ctx=a.ctx).build()
    many = synthetic.make_scene(12000, 4, 4, layout="shell", s_range=(0.03, 0.06), empty_frac=0.5)
    cam = synthetic.look_at_camera((0.4, 0.3, -3.0), 72, 56, 72.0)
    d = Dev(many, synthetic.make_rays([cam], 1.0, 5.0, 0.01), ctx=a.ctx).build()
    empty = synthetic.Scene(t=sc.t[:0], q=sc.q[:0], s=sc.s[:0], payload=sc.payload[:0], M=sc.M)
    er = rays_from(rays.o, rays.d, rays.t_near, rays.t_far, rays.dt, bg=(0.25, 0.5, 0.75))
    e = Dev(empty, er, ctx=a.ctx).build()
    return [a, a, b, c, d, e, a]


def test_static_entry_point_matches_allocating_path():
    torch.cuda.set_device(0)
    scenes = _scenes()
    refs = {id(dv): dv.render()[0] for dv in scenes}
    status = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    for dv in scenes:  # two calls in a row, then other scenes, sizes, payload types
        ref = refs[id(dv)]
        out = torch.full_like(ref, float("nan"))
        _static_render(dv, out, status)
        assert status.item() == 0
        assert torch.isfinite(out).all()
        # the same kernels on the same inputs: agreement to FP32 summation order
        assert (out - ref).abs().max().item() <= 1e-5
        if dv.scene.n == 0:  # an empty scene after full ones: exactly the background
            bg = torch.tensor(dv.rays.bg, dtype=torch.float32, device=DEV)
            assert torch.equal(out[:, :3], bg.expand_as(out[:, :3]))
            assert torch.count_nonzero(out[:, 3]).item() == 0
        elif dv.scene.n == 12000:
            assert out[:, 3].max().item() > 0  # the many-primitive scene is in view


def test_static_entry_point_allocates_nothing():
    """After one call of each scene (which also loads the kernels it needs), another round
    of calls leaves the device's free memory unchanged."""
    torch.cuda.set_device(0)
    scenes = _scenes()
    outs = [torch.empty((dv.rays.n, 4), dtype=torch.float32, device=DEV) for dv in scenes]
    status = torch.zeros((1,), dtype=torch.int32, device=DEV)
    for dv, out in zip(scenes, outs):
        _static_render(dv, out, status)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        for dv, out in zip(scenes, outs):
            _static_render(dv, out, status)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_entry_point_rejects_too_many_primitives():
    torch.cuda.set_device(0)
    n = 16384 + 1
    sc = synthetic.make_scene(n, 2, 0, s_range=(0.01, 0.02))
    rays = synthetic.make_config("tiny_8x8^3_64x64", 0)[1]
    dv = Dev(sc, rays)
    out = torch.zeros((rays.n, 4), dtype=torch.float32, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = B.lib().mvp_raymarch_fwd_static(ctypes.byref(dv.prims), ctypes.byref(dv.rs),
                                         ctypes.c_void_p(out.data_ptr()), None, stream)
    assert st == B.MVP_ERR_INVALID_ARG
    assert b"MVP_STATIC_MAX_PRIMS" in B.lib().mvp_last_error()
    assert torch.count_nonzero(out).item() == 0


# A process without PyTorch (its allocator would keep addresses that a device reset
# frees): render, reset the device, render again into fresh buffers. The entry point
# must notice that the device's context was re-created and look its array up again.
_RESET_CHILD = r"""
import ctypes, sys
import numpy as np
sys.path[:0] = [{root!r}, {tests!r}]
import synthetic
from paper_2103_01954_gb300 import binding as B

rt = ctypes.CDLL("libcudart.so.13")
drv = ctypes.CDLL("libcuda.so.1")
H2D, D2H = 1, 2

def ctx_id():
    c = ctypes.c_void_p()
    assert drv.cuCtxGetCurrent(ctypes.byref(c)) == 0 and c.value
    i = ctypes.c_ulonglong()
    assert drv.cuCtxGetId(c, ctypes.byref(i)) == 0
    return i.value

def upload(a):
    a = np.ascontiguousarray(a)
    p = ctypes.c_void_p()
    assert rt.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(max(a.nbytes, 16))) == 0
    assert rt.cudaMemcpy(p, a.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(a.nbytes), H2D) == 0
    return p

def render(sc, rays):
    t, q, s, pl = (upload(x) for x in (sc.t, sc.q, sc.s, sc.payload))
    o, d = upload(rays.o), upload(rays.d)
    out = upload(np.zeros((rays.n, 4), np.float32))
    status = upload(np.full(1, -1, np.int32))
    prims = B.mvp_prims(n=sc.n, M=sc.M, dtype=B.MVP_F32, reserved=0, t=t, q=q, s=s, payload=pl)
    rs = B.mvp_rays(n=rays.n, o=o, d=d, t_near=rays.t_near, t_far=rays.t_far, dt=rays.dt, eps_early=0.0,
                    width=rays.width, height=rays.height, flags=0)
    B.check(B.lib().mvp_raymarch_fwd_static(ctypes.byref(prims), ctypes.byref(rs), out, status, None), "static")
    assert rt.cudaDeviceSynchronize() == 0
    img = np.zeros((rays.n, 4), np.float32)
    st = np.zeros(1, np.int32)
    assert rt.cudaMemcpy(img.ctypes.data_as(ctypes.c_void_p), out, ctypes.c_size_t(img.nbytes), D2H) == 0
    assert rt.cudaMemcpy(st.ctypes.data_as(ctypes.c_void_p), status, ctypes.c_size_t(4), D2H) == 0
    return img, int(st[0])

assert rt.cudaSetDevice(0) == 0
sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 0)
a, sa = render(sc, rays)
before = ctx_id()
assert rt.cudaDeviceReset() == 0
assert rt.cudaFree(None) == 0  # re-create the primary context
after = ctx_id()
if after == before:
    print("CONTEXT ID UNCHANGED")
    sys.exit(3)
b, sb = render(sc, rays)
assert sa == 0 and sb == 0, (sa, sb)
assert np.array_equal(a, b), float(np.abs(a - b).max())
assert a[:, 3].max() > 0
print("RESET OK")
"""


def test_static_entry_point_after_device_reset():
    code = _RESET_CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES=os.environ.get("CUDA_VISIBLE_DEVICES", str(torch.cuda.current_device())))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0 and "RESET OK" in r.stdout, (r.returncode, r.stdout[-2000:], r.stderr[-2000:])
