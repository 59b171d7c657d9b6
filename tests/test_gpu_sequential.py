"""GPU parity of the sequential blending mode (MVP_BLEND_SEQUENTIAL: the primitives that
share a ray's saturating sample blended one by one in BVH order, Sec. 3.2.2) against
the oracle's matching mode, on the same seeded inputs.

Bar: as for the default rule, at least 99.9% of pixel channels within 2e-4 and all
within 1e-2 of the FP64 oracle; in addition, on every pixel where the two rules differ
by more than 1e-3, the GPU image must sit with the sequential oracle, not the summed
one (so the flag demonstrably changes the blend).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic
from helpers import concat_scenes, rays_from, single_box

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from gpu_util import DEV, Dev, image_parity  # noqa: E402
from paper_2103_01954_gb300 import binding as B  # noqa: E402
from paper_2103_01954_gb300 import torch_ops as T  # noqa: E402

F32M = oracle.MODE_PRUNED | oracle.MEMBER_F32
SEQM = F32M | oracle.SEQUENTIAL


def _sequential(dv):
    dv.rs = T.rays_struct(dv.o, dv.d, sequential=True, **dv.params)
    return dv


def _check(gpu, sc, rays, label):
    seq = oracle.render(sc, rays, SEQM)["rgba"]
    summ = oracle.render(sc, rays, F32M)["rgba"]
    st = image_parity(gpu, seq)
    print(label, st)
    assert st["frac_2e-4"] >= 0.999 and st["max"] <= 1e-2, (label, st)
    differ = np.abs(seq - summ).max(1) > 1e-3
    if differ.any():
        e_seq = np.abs(gpu[differ] - seq[differ]).max(1)
        e_sum = np.abs(gpu[differ] - summ[differ]).max(1)
        assert (e_seq < e_sum).mean() >= 0.99, (label, int(differ.sum()))
    return int(differ.sum())


@pytest.mark.parametrize("cfg", ["tiny_8x8^3_64x64", "small_512x8^3_96x128", "small_4096x16^3_83x128"])
def test_sequential_matches_oracle(cfg):
    sc, rays, _ = synthetic.make_config(cfg, 0)
    dv = _sequential(Dev(sc, rays)).build()
    out, _ = dv.render()
    n = _check(out.cpu().numpy(), sc, rays, cfg)
    assert n > 0  # the scene has saturating samples shared by several primitives


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_sequential_reduced_precision_payload(dtype):
    """BF16 / FP16 storage: parity against the oracle on the dequantised payload."""
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 2)
    dv = _sequential(Dev(sc, rays, payload_dtype=dtype)).build()
    out, _ = dv.render()
    deq = torch.from_numpy(sc.payload).to(dtype).float().numpy()
    sc2 = synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, payload=deq, M=sc.M)
    _check(out.cpu().numpy(), sc2, rays, str(dtype))


def test_sequential_pair_closed_form():
    """Two constant boxes whose centres differ only in x: the one at lower x (lower
    Morton key) blends first at the saturating sample, whichever index it has."""
    dt, aA, aB = 0.01, 17.0, 19.0
    cA, cB = np.float32([0.9, 0.1, 0.2]).astype(np.float64), np.float32([0.1, 0.7, 0.4]).astype(np.float64)
    rays = rays_from([0, 0, -3], np.repeat([[0.0, 0.0, 1.0]], 64, 0), 0.0037, 6.0, dt)
    rem = 1.0 - 2 * dt * (aA + aB)
    expect = 2 * dt * (aA * cA + aB * cB) + cA * dt * aA + cB * (rem - dt * aA)
    for order in ((0, 1), (1, 0)):
        boxes = [single_box(M=3, alpha=aA, rgb=cA, t=(-0.05, 0, 0)), single_box(M=3, alpha=aB, rgb=cB, t=(0.05, 0, 0))]
        sc = concat_scenes(boxes[order[0]], boxes[order[1]])
        out, _ = _sequential(Dev(sc, rays)).build().render()
        got = out.cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got[:, :3], np.broadcast_to(expect, (64, 3)), atol=2e-6)
        assert np.all(got[:, 3] == 1.0)


@pytest.mark.parametrize("n", [12, 40])
def test_sequential_dense_overlap(n):
    """n opaque boxes stacked on one another: every saturating sample holds all of them."""
    rng = np.random.default_rng(n)
    base = single_box(M=3, alpha=1.0, s=(0.5, 0.5, 0.5))
    payload = np.repeat(base.payload, n, 0)
    payload[..., :3] = rng.uniform(0.0, 1.0, (n, 1, 1, 1, 3)).astype(np.float32)
    payload[..., 3] = rng.uniform(0.5, 1.5, (n, 3, 3, 3)).astype(np.float32)
    t = rng.uniform(-0.05, 0.05, (n, 3)).astype(np.float32)
    sc = synthetic.Scene(t=t, q=synthetic.random_unit_quaternions(rng, n), s=np.repeat(base.s, n, 0),
                         payload=payload, M=3)
    cam = synthetic.look_at_camera((0.3, -0.2, -3.0), 20, 12, 16.0)
    rays = synthetic.make_rays([cam], 1.0, 5.0, 0.02)
    out, _ = _sequential(Dev(sc, rays)).build().render()
    assert _check(out.cpu().numpy(), sc, rays, f"dense{n}") > 0


def test_sequential_static_entry_point_and_flags():
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 1)
    dv = _sequential(Dev(sc, rays)).build()
    ref, _ = dv.render()
    out = torch.full_like(ref, float("nan"))
    status = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    B.check(B.lib().mvp_raymarch_fwd_static(ctypes.byref(dv.prims), ctypes.byref(dv.rs),
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                                            stream), "mvp_raymarch_fwd_static")
    torch.cuda.synchronize()
    assert status.item() == 0
    assert (out - ref).abs().max().item() <= 1e-5
    # unknown flag bits are refused
    bad = T.rays_struct(dv.o, dv.d, **dv.params)
    bad.flags = 6
    with pytest.raises(B.MVPError):
        T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, bad)


@pytest.mark.parametrize("cfg,seed", [("diff_small_64x8^3_2x48x40", 1), ("diff_small_64x8^3_2x48x40", 3),
                                      ("small_512x8^3_96x128", 0)])
def test_sequential_adjoint_matches_oracle(cfg, seed):
    """The adjoint of the sequential rule (forward and backward with the flag): payload
    and pose gradients within 1e-3 of the oracle's sequential adjoint, and different
    from the summed rule's where the rule matters."""
    from helpers import zero_boundary

    sc, rays, _ = synthetic.make_config(cfg, seed)
    sc = zero_boundary(sc)
    dv = _sequential(Dev(sc, rays)).build()
    out, saved = T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, dv.rs, want_saved=True)
    g = np.random.default_rng(seed + 9).standard_normal((rays.n, 4))
    # Near-ties of the saturation decision are kinks of the image: FP32 (kernel) and FP64
    # (oracle) may take them on different sides (the saturating sample, or which
    # primitive is clamped in it) and then differentiate different pieces. Rays whose
    # discrete decisions differ are left out of the loss; they must be rare.
    sv = saved.cpu().numpy().view(np.int32).reshape(rays.n, 8)
    ref = oracle.render(sc, rays, SEQM)
    keys = oracle.morton_keys(sc.t)[1]
    rank = np.empty(sc.n, np.int64)
    rank[(np.sort(keys) & 0xffffffff).astype(np.int64)] = np.arange(sc.n)
    clamped = ref["i_clamp"] >= 0
    orc_rank = np.where(ref["clamp_k"] >= 0, rank[np.maximum(ref["clamp_k"], 0)], 0x7fffffff)
    tie = (sv[:, 5] != ref["i_clamp"]) | (clamped & (sv[:, 6] != orc_rank))
    assert tie.mean() <= 0.005, tie.mean()
    g[tie] = 0.0
    gt = torch.from_numpy(g.astype(np.float32)).to(DEV)
    gp = torch.zeros(dv.payload.shape, dtype=torch.float32, device=DEV)
    g_t, g_q, g_s = torch.zeros_like(dv.t), torch.zeros_like(dv.q), torch.zeros_like(dv.s)
    T.raymarch_bwd(dv.ctx, dv.prims, dv.bvh, dv.rs, saved, gt, gp, g_t, g_q, g_s)
    dv.ctx.sync()
    g64 = g.astype(np.float32).astype(np.float64)
    R = oracle.backward(sc, rays, g64, SEQM)
    Rs = oracle.backward(sc, rays, g64, F32M)
    for key, val in (("g_payload", gp), ("g_t", g_t), ("g_q", g_q), ("g_s", g_s)):
        v = val.cpu().numpy().astype(np.float64)
        rel = np.abs(v - R[key]).max() / max(np.abs(R[key]).max(), 1e-30)
        assert rel <= 1e-3, (key, rel)
    assert np.abs(R["g_payload"] - Rs["g_payload"]).max() > 1e-2 * np.abs(R["g_payload"]).max()
