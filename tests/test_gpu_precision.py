"""Reduced-precision payloads (BF16, FP16; interpolation and compositing stay FP32).

The conversion kernel is byte work: bit-exact against PyTorch's CPU round-to-nearest
conversion. The march on a converted payload is held to the FP32 parity bar against
the oracle run on the same (dequantised, exactly representable) values; the error
against the oracle on the original FP32 payload is reported per dtype.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from helpers import rays_from

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from gpu_util import DEV, Dev, image_parity  # noqa: E402
from paper_2103_01954_gb300 import torch_ops as T  # noqa: E402

F32M = oracle.MODE_PRUNED | oracle.MEMBER_F32
F64M = oracle.MODE_PRUNED | oracle.MEMBER_F64
DTYPES = [torch.bfloat16, torch.float16]


@pytest.mark.parametrize("dtype", DTYPES)
def test_pack_bit_exact(dtype):
    rng = np.random.default_rng(0)
    x = rng.standard_normal(4 * 1000 + 3).astype(np.float32) * 10  # ragged tail
    x[:8] = [0.0, -0.0, 1e-30, 65504.0, 1e5, -3.0e38, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9]
    ctx = T.Context(0)
    g = T.pack_payload(ctx, torch.from_numpy(x).to(DEV), dtype)
    ref = torch.from_numpy(x).to(dtype)
    torch.cuda.synchronize()
    assert torch.equal(g.cpu().view(torch.int16), ref.view(torch.int16))


def _report(cfg, dtype, e, st):
    """Max and 99.9th percentile over pixel channels of the error against the FP64
    oracle on the FP32 payload (the configs' precision figure), printed and kept for the
    session summary."""
    from parity_rules import REPORT

    r = {"max": float(e.max()), "p999": float(np.quantile(e, 0.999)), "vs_dequantised_max": float(st["max"])}
    print(f"{cfg} {dtype}: vs FP64 oracle on the FP32 payload max {r['max']:.3e} p99.9 {r['p999']:.3e}; "
          f"vs the oracle on the dequantised payload max {r['vs_dequantised_max']:.3e}")
    REPORT.append(("precision", f"{cfg} {str(dtype).replace('torch.', '')}", r))


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("cfg", ["small_512x8^3_96x128", "small_4096x16^3_83x128"])
def test_reduced_precision_payload(dtype, cfg):
    sc, rays, _ = synthetic.make_config(cfg, 0)
    dv = Dev(sc, rays, payload_dtype=dtype).build()
    out, _ = dv.render()
    o = out.cpu().numpy()
    deq = torch.from_numpy(sc.payload).to(dtype).float().numpy()
    sc_q = synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, payload=deq, M=sc.M)
    ref_q = oracle.render(sc_q, rays, F32M)["rgba"]
    st = image_parity(o, ref_q)
    assert st["frac_2e-4"] >= 0.999 and st["max"] <= 1e-2, st
    # the whole error of the stored precision: against the FP64 oracle on the original FP32 payload
    ref64 = oracle.render(sc, rays, F64M)["rgba"]
    e = np.abs(o - ref64)
    _report(cfg, dtype, e, st)
    assert e.max() < 0.1


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("cfg", ["paper_4096x16^3_667x1024", "sweep_32768x8^3_667x1024"])
def test_reduced_precision_full_scale_sampled(dtype, cfg):
    """The benchmark frames with BF16/FP16 payloads on 2000 sampled pixels: FP32 parity
    against the oracle on the dequantised payload, and the error against the FP64
    oracle on the original FP32 payload reported (max and 99.9th percentile over
    channels)."""
    sc, rays, _ = synthetic.make_config(cfg, 0)
    dv = Dev(sc, rays, payload_dtype=dtype).build()
    out, _ = dv.render()
    sel = np.random.default_rng(2).choice(rays.n, 2000, replace=False)
    sub = rays_from(rays.o[sel], rays.d[sel], rays.t_near, rays.t_far, rays.dt)
    deq = torch.from_numpy(sc.payload).to(dtype).float().numpy()
    ref_q = oracle.render(synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, payload=deq, M=sc.M), sub, F32M)["rgba"]
    o = out.cpu().numpy()[sel]
    st = image_parity(o, ref_q)
    assert st["frac_2e-4"] >= 0.999 and st["max"] <= 1e-2, st
    # the whole error of the stored precision: against the FP64 oracle on the original FP32 payload
    ref64 = oracle.render(sc, sub, F64M)["rgba"]
    e = np.abs(o - ref64)
    _report(cfg, dtype, e, st)
    assert e.max() < 0.1


def test_bf16_backward_runs_and_matches_dequantised_oracle():
    sc, rays, _ = synthetic.make_config("diff_small_64x8^3_2x48x40", 0)
    dv = Dev(sc, rays, payload_dtype=torch.bfloat16).build()
    out, saved = T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, dv.rs, want_saved=True)
    g = np.random.default_rng(0).standard_normal((rays.n, 4)).astype(np.float32)
    gp = torch.zeros(dv.payload.shape, dtype=torch.float32, device=DEV)
    T.raymarch_bwd(dv.ctx, dv.prims, dv.bvh, dv.rs, saved, torch.from_numpy(g).to(DEV), gp)
    dv.ctx.sync()
    deq = torch.from_numpy(sc.payload).to(torch.bfloat16).float().numpy()
    R = oracle.backward(synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, payload=deq, M=sc.M), rays,
                        g.astype(np.float64), F32M)
    ref = R["g_payload"]
    assert np.abs(gp.cpu().numpy() - ref).max() / np.abs(ref).max() <= 1e-3
