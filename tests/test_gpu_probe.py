"""The roofline probe (mvp_gather_probe) performs every access it counts.

Loads: on an all-ones payload the sink receives 4 x (voxel accesses) exactly (each
warp's partial sum is a multiple of 4096 and the total stays exact in FP32).
Reductions: the gradient array's total is (accesses) x (1 + 2 + 3 + 4) 1e-3.
"""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from gpu_util import DEV  # noqa: E402
from paper_2103_01954_gb300 import binding as B  # noqa: E402


def _probe(payload, dtype, n, M, mode, footprint, steps, grad=None, sink=None):
    acc = ctypes.c_int64(0)
    st = B.lib().mvp_gather_probe(ctypes.c_void_p(payload.data_ptr()) if payload is not None else None, dtype, n, M,
                                  mode, footprint, steps,
                                  ctypes.c_void_p(grad.data_ptr()) if grad is not None else None,
                                  ctypes.c_void_p(sink.data_ptr()) if sink is not None else None, ctypes.byref(acc),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, acc.value


@pytest.mark.parametrize("dtype,tdt", [(B.MVP_F32, torch.float32), (B.MVP_BF16, torch.bfloat16),
                                       (B.MVP_F16, torch.float16)])
@pytest.mark.parametrize("footprint", [0, 1])
@pytest.mark.parametrize("mode,per", [(0, 1), (2, 2), (3, 4), (4, 1)])
def test_probe_loads_every_access(dtype, tdt, footprint, mode, per):
    n, M = 200, 16
    payload = torch.ones((n, M, M, M, per, 4), dtype=tdt, device=DEV)
    sink = torch.zeros(1, dtype=torch.float32, device=DEV)
    st, acc = _probe(payload, dtype, n, M, mode, footprint, 8, sink=sink)
    B.check(st, "probe")
    torch.cuda.synchronize()
    assert acc > 0 and acc % 8 == 0
    assert sink.item() == 4.0 * acc


@pytest.mark.parametrize("M", [8, 16, 32])
def test_probe_reduces_every_access(M):
    n = 64
    grad = torch.zeros((n, M, M, M, 4), dtype=torch.float32, device=DEV)
    st, acc = _probe(None, B.MVP_F32, n, M, 1, 1, 4, grad=grad)
    B.check(st, "probe")
    torch.cuda.synchronize()
    total = grad.double().sum().item()
    assert abs(total - acc * 0.010) <= 1e-4 * acc * 0.010
    # every corner of a cell lies inside its primitive's grid: the last voxel is reachable
    assert grad.abs().sum().item() > 0


@pytest.mark.parametrize("blocks", [3, 5])
@pytest.mark.parametrize("footprint", [0, 1])
def test_probe_at_the_kernels_residency_counts_every_access(blocks, footprint):
    """mode | (blocks << 8): 4-warp blocks at the march kernels' residency; loads and
    reductions are still all performed, and the access count is that launch's."""
    n, M = 200, 16
    payload = torch.ones((n, M, M, M, 4), dtype=torch.float32, device=DEV)
    sink = torch.zeros(1, dtype=torch.float32, device=DEV)
    st, acc = _probe(payload, B.MVP_F32, n, M, 0 | (blocks << 8), footprint, 8, sink=sink)
    B.check(st, "probe at residency")
    torch.cuda.synchronize()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert acc == sms * blocks * 128 * 8 * 8
    assert sink.item() == 4.0 * acc
    grad = torch.zeros((64, M, M, M, 4), dtype=torch.float32, device=DEV)
    st, acc = _probe(None, B.MVP_F32, 64, M, 1 | (blocks << 8), footprint, 4, grad=grad)
    B.check(st, "reductions at residency")
    torch.cuda.synchronize()
    assert abs(grad.double().sum().item() - acc * 0.010) <= 1e-4 * acc * 0.010


def test_probe_rejects_bad_arguments():
    sink = torch.zeros(1, dtype=torch.float32, device=DEV)
    p = torch.ones((4, 8, 8, 8, 4), dtype=torch.float32, device=DEV)
    assert _probe(p, B.MVP_F32, 0, 8, 0, 0, 4, sink=sink)[0] == B.MVP_ERR_INVALID_ARG
    assert _probe(p, B.MVP_F32, 4, 1, 0, 0, 4, sink=sink)[0] == B.MVP_ERR_INVALID_ARG
    assert _probe(p, B.MVP_F32, 4, 8, 5, 0, 4, sink=sink)[0] == B.MVP_ERR_INVALID_ARG
    assert _probe(p, B.MVP_F32, 4, 8, 2 | (5 << 8), 0, 4, sink=sink)[0] == B.MVP_ERR_INVALID_ARG  # layouts: full only
    assert _probe(p, B.MVP_F32, 4, 8, 0 | (17 << 8), 0, 4, sink=sink)[0] == B.MVP_ERR_INVALID_ARG
    assert _probe(p, B.MVP_F32, 4, 8, 1 << 16, 0, 4, sink=sink)[0] == B.MVP_ERR_INVALID_ARG
    assert _probe(p, B.MVP_F32, 4, 8, 0, 0, 4)[0] == B.MVP_ERR_INVALID_ARG  # no sink
    assert _probe(None, B.MVP_F32, 4, 8, 1, 0, 4)[0] == B.MVP_ERR_INVALID_ARG  # no grad
    v = p.view(-1)[1:]  # 4-byte offset: misaligned for 16-byte voxels
    assert _probe(v, B.MVP_F32, 4, 8, 0, 0, 4, sink=sink)[0] == B.MVP_ERR_INVALID_ARG
    v = p.view(-1)[4:]  # 16-byte aligned, but the pair layout's 32-byte elements are not
    assert _probe(v, B.MVP_F32, 2, 8, 2, 0, 4, sink=sink)[0] == B.MVP_ERR_INVALID_ARG
