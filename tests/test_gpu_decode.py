"""GPU decode-side epilogues (opacity fade fused with the payload conversion,
axis-angle rotations and their gradient, volume prior) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from oracle import decode as D

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from gpu_util import DEV, Dev, image_parity  # noqa: E402
from paper_2103_01954_gb300 import binding as B  # noqa: E402
from paper_2103_01954_gb300 import torch_ops as T  # noqa: E402

F32M = oracle.MODE_PRUNED | oracle.MEMBER_F32
ULP = {torch.float32: 2.0 ** -23, torch.bfloat16: 2.0 ** -8, torch.float16: 2.0 ** -11}


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("M,n", [(8, 37), (16, 5), (3, 1000), (32, 2)])
def test_fade_matches_oracle(dtype, M, n):
    ctx = T.Context(0)
    rng = np.random.default_rng(M * 100 + n)
    p = rng.uniform(0.0, 4.0, (n, M, M, M, 4)).astype(np.float32)
    g = T.fade_payload(ctx, torch.from_numpy(p).to(DEV), dtype, 8.0, 8)
    ctx.sync()
    got = g.float().cpu().numpy().astype(np.float64)
    ref = D.fade_payload(p, 8.0, 8)
    # FP32 evaluation of W: the coordinate (2i/(M-1) - 1) and its 8th power carry a few
    # units of 2^-23 each, which exp(-alpha * sum of three powers) turns into a relative
    # error of at most alpha * 3 * beta * 4 * 2^-23 = 9.2e-5 (alpha = beta = 8; |x| <= 1); then
    # one rounding to the stored type
    # (FP16 keeps absolute steps of 2^-24 below its normal range: half of that more)
    floor = 2.0 ** -25 if dtype == torch.float16 else 0.0
    tol = (ULP[dtype] + 8.0 * 3 * 8 * 4 * ULP[torch.float32]) * np.abs(ref) + floor + 1e-30
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / (np.abs(ref) + 1e-30))
    assert np.array_equal(got[..., :3], torch.from_numpy(p[..., :3]).to(dtype).double().numpy())


def test_fade_in_place_fp32_and_overlap_rejected():
    ctx = T.Context(0)
    p = torch.rand((4, 6, 6, 6, 4), device=DEV)
    ref = D.fade_payload(p.cpu().numpy(), 2.0, 4)
    T.fade_payload(ctx, p, torch.float32, 2.0, 4, out=p)  # in place
    ctx.sync()
    assert np.allclose(p.cpu().numpy(), ref, rtol=1e-6)
    # a BF16 output over its own FP32 input is refused before any launch
    st = B.lib().mvp_fade_payload(ctx.handle, T._ptr(p), T._ptr(p), 4, 6, B.MVP_BF16, 2.0, 4, None)
    assert st == B.MVP_ERR_INVALID_ARG
    st = B.lib().mvp_fade_payload(ctx.handle, T._ptr(p), T._ptr(p), 4, 1, B.MVP_F32, 2.0, 4, None)
    assert st == B.MVP_ERR_INVALID_ARG  # M < 2


def test_faded_payload_renders_like_the_oracle():
    """The fused fade + BF16 conversion feeds the march: image equal to the oracle on
    the same (faded, dequantised) payload."""
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 0)
    ctx = T.Context(0)
    pb = T.fade_payload(ctx, torch.from_numpy(sc.payload).to(DEV), torch.bfloat16, 8.0, 8)
    dv = Dev(sc, rays, ctx=ctx)
    dv.payload = pb
    dv.prims = T.prims_struct(dv.t, dv.q, dv.s, pb)
    out, _ = dv.build().render()
    deq = pb.float().cpu().numpy()
    ref = oracle.render(synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, payload=deq, M=sc.M), rays, F32M)["rgba"]
    st = image_parity(out.cpu().numpy(), ref)
    assert st["frac_2e-4"] >= 0.999 and st["max"] <= 1e-2, st


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("M,n,alpha", [(8, 37, 8.0), (16, 5, 8.0), (3, 1000, 0.0), (32, 2, 2.0)])
def test_assemble_matches_oracle(dtype, M, n, alpha):
    """A view's payload from its colour and the shared opacity: colour channels are the
    input rounded once to the stored type; opacity within the fade's FP32 bound."""
    ctx = T.Context(0)
    rng = np.random.default_rng(M * 10 + n)
    rgb = rng.uniform(0.0, 1.0, (n, M, M, M, 3)).astype(np.float32)
    op = rng.uniform(0.0, 4.0, (n, M, M, M)).astype(np.float32)
    g = T.assemble_payload(ctx, torch.from_numpy(rgb).to(DEV), torch.from_numpy(op).to(DEV), dtype, alpha, 8)
    ctx.sync()
    got = g.float().cpu().numpy().astype(np.float64)
    ref = D.assemble_payload(rgb, op, alpha, 8)
    assert np.array_equal(got[..., :3], torch.from_numpy(rgb).to(dtype).double().numpy())
    floor = 2.0 ** -25 if dtype == torch.float16 else 0.0
    tol = (ULP[dtype] + alpha * 3 * 8 * 4 * ULP[torch.float32]) * np.abs(ref[..., 3]) + floor + 1e-30
    assert np.all(np.abs(got[..., 3] - ref[..., 3]) <= tol)
    if alpha == 0.0:  # no fade: the opacity is only rounded to the stored type
        assert np.array_equal(got[..., 3], torch.from_numpy(op).to(dtype).double().numpy())


def test_assemble_rejects_overlap_and_misalignment():
    ctx = T.Context(0)
    buf = torch.zeros(4 * 6 ** 3 * 4 + 8, device=DEV)
    rgb = torch.rand((4, 6, 6, 6, 3), device=DEV)
    op = torch.rand((4, 6, 6, 6), device=DEV)
    lib = B.lib()
    # destination over the colour input
    st = lib.mvp_assemble_payload(ctx.handle, T._ptr(rgb), T._ptr(op), T._ptr(rgb), 4, 6, B.MVP_BF16, 8.0, 8, None)
    assert st == B.MVP_ERR_INVALID_ARG
    # FP32 destination not 16-byte aligned
    st = lib.mvp_assemble_payload(ctx.handle, T._ptr(rgb), T._ptr(op), buf.data_ptr() + 4, 4, 6, B.MVP_F32, 8.0, 8,
                                  None)
    assert st == B.MVP_ERR_INVALID_ARG
    st = lib.mvp_assemble_payload(ctx.handle, T._ptr(rgb), T._ptr(op), T._ptr(buf), 4, 6, B.MVP_F32, 8.0, 8, None)
    assert st == B.MVP_OK
    ctx.sync()


def test_view_payloads_render_like_the_oracle():
    """Two views' payloads assembled on the device (BF16, faded) render as the oracle
    renders the same dequantised payloads, and the two views' images differ."""
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 3)
    ctx = T.Context(0)
    op = torch.from_numpy(np.ascontiguousarray(sc.payload[..., 3])).to(DEV)
    imgs = []
    for view in ((0.0, 0.0, 1.0), (1.0, 0.0, 0.0)):
        rgb = synthetic.view_colors(sc, view, seed=3)
        pb = T.assemble_payload(ctx, torch.from_numpy(rgb).to(DEV), op, torch.bfloat16, 8.0, 8)
        dv = Dev(sc, rays, ctx=ctx)
        dv.payload = pb
        dv.prims = T.prims_struct(dv.t, dv.q, dv.s, pb)
        out, _ = dv.build().render()
        deq = pb.float().cpu().numpy()
        ref = oracle.render(synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, payload=deq, M=sc.M), rays, F32M)["rgba"]
        st = image_parity(out.cpu().numpy(), ref)
        assert st["frac_2e-4"] >= 0.999 and st["max"] <= 1e-2, st
        imgs.append(out.cpu().numpy())
    assert np.abs(imgs[0] - imgs[1]).max() > 1e-2


def test_axis_angle_and_gradient_match_oracle():
    ctx = T.Context(0)
    rng = np.random.default_rng(3)
    r = (rng.standard_normal((500, 3)) * rng.uniform(0, 3.0, (500, 1))).astype(np.float32)
    r[:4] = [[0, 0, 0], [1e-6, 0, 0], [3e-4, -2e-4, 1e-4], [0, 0, 3.1]]
    rt = torch.from_numpy(r).to(DEV)
    q = T.axis_angle_to_quat(ctx, rt)
    g = rng.standard_normal((500, 4)).astype(np.float32)
    gr = torch.full((500, 3), 0.25, device=DEV)  # accumulates
    T.axis_angle_backward(ctx, rt, torch.from_numpy(g).to(DEV), gr)
    ctx.sync()
    assert np.allclose(q.cpu().numpy(), D.axis_angle_to_quat(r), atol=2e-7)
    assert np.allclose(gr.cpu().numpy() - 0.25, D.axis_angle_vjp(r, g), atol=2e-6)


def test_axis_angle_feeds_the_march():
    """Rendering with q from axis-angle equals rendering with the oracle's quaternion."""
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 1)
    rng = np.random.default_rng(4)
    r = (rng.standard_normal((sc.t.shape[0], 3)) * 1.5).astype(np.float32)
    ctx = T.Context(0)
    q = T.axis_angle_to_quat(ctx, torch.from_numpy(r).to(DEV)).cpu().numpy()
    sc2 = synthetic.Scene(t=sc.t, q=q, s=sc.s, payload=sc.payload, M=sc.M)
    out, _ = Dev(sc2, rays, ctx=ctx).build().render()
    ref = oracle.render(sc2, rays, F32M)["rgba"]
    st = image_parity(out.cpu().numpy(), ref)
    assert st["frac_2e-4"] >= 0.999 and st["max"] <= 1e-2, st


def test_volume_prior_matches_oracle():
    ctx = T.Context(0)
    rng = np.random.default_rng(5)
    s = rng.uniform(0.02, 0.3, (3000, 3)).astype(np.float32)
    st = torch.from_numpy(s).to(DEV)
    g0 = 1.0e-3  # the call accumulates into g_s
    gs = torch.full((3000, 3), g0, device=DEV)
    loss, _ = T.volume_prior(ctx, st, 0.01, gs)
    ctx.sync()
    ref_loss, ref_g = D.volume_prior(s, 0.01)
    assert np.isclose(loss.item(), ref_loss, rtol=1e-5)
    # FP32 products and one FP32 addition to g0
    assert np.allclose(gs.cpu().numpy().astype(np.float64), ref_g + np.float32(g0), rtol=2e-6, atol=1e-10)
