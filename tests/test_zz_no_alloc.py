"""The allocation-free render entry point (mvp_raymarch_fwd_static).

It exists for callers that cannot allocate device memory (a plug-in inside an
application that owns the device allocator, a frame loop that must not stall on
cudaMalloc/cudaFree). It keeps its BVH in a fixed device array inside the library,
so it must give the same image as the allocating path (mvp_build_bvh +
mvp_raymarch_fwd) on every call, including a call that follows another scene.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from gpu_util import DEV, Dev  # noqa: E402
from paper_2103_01954_gb300 import binding as B  # noqa: E402


def _static_render(dv, out, status):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = B.lib().mvp_raymarch_fwd_static(ctypes.byref(dv.prims), ctypes.byref(dv.rs),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(status.data_ptr()), stream)
    B.check(st, "mvp_raymarch_fwd_static")
    torch.cuda.synchronize()


def test_static_entry_point_matches_allocating_path():
    torch.cuda.set_device(0)
    a = Dev(*synthetic.make_config("small_4096x16^3_83x128", 0)[:2]).build()
    b = Dev(*synthetic.make_config("small_512x8^3_96x128", 1)[:2], ctx=a.ctx).build()
    ref_a, _ = a.render()
    ref_b, _ = b.render()
    status = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    for dv, ref in ((a, ref_a), (a, ref_a), (b, ref_b), (a, ref_a)):  # two calls in a row, then another scene
        out = torch.full_like(ref, float("nan"))
        _static_render(dv, out, status)
        assert status.item() == 0
        assert torch.isfinite(out).all()
        # the same kernels on the same inputs: agreement to FP32 summation order
        assert (out - ref).abs().max().item() <= 1e-5


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
