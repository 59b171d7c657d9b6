"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Bars: BVH keys, sort order, tree and hit lists bit-exact (integer / index work;
the FP32 membership decision is reproduced by the oracle with the same operation
order). Images: at least 99.9% of pixel channels within 2e-4 and all within 1e-2 of
the FP64 oracle. Evaluation counts: exact except where the FP32 and FP64
accumulations reach T = 1 on different samples.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from helpers import concat_scenes, rays_from, single_box

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from gpu_util import Dev, image_parity  # noqa: E402
from paper_2103_01954_gb300 import binding as B  # noqa: E402
from paper_2103_01954_gb300 import torch_ops as T  # noqa: E402

F32M = oracle.MODE_PRUNED | oracle.MEMBER_F32


def _check_image(gpu, ref, label=""):
    st = image_parity(gpu, ref)
    print(label, st)
    assert st["frac_2e-4"] >= 0.999, (label, st)
    assert st["max"] <= 1e-2, (label, st)
    return st


# --------------------------------------------------------------------------- BVH
def _scene_n(n, seed=0, dup=False):
    if n == 0:
        sc = synthetic.make_scene(1, 4, seed)
        return synthetic.Scene(t=sc.t[:0], q=sc.q[:0], s=sc.s[:0], payload=sc.payload[:0], M=4)
    sc = synthetic.make_scene(n, 4, seed, layout="shell", s_range=(0.02, 0.05), empty_frac=0.5)
    if dup == "cluster":  # 200 equal centres: one Morton code for all of them
        sc.t[:200] = sc.t[0]
    elif dup and n > 20:
        sc.t[10:20] = sc.t[3]
    return sc


@pytest.mark.parametrize("n,dup", [(1, False), (2, False), (3, False), (50, True), (513, False), (1000, "cluster"),
                                   (4096, "cluster"), (5000, True), (8192, True), (8193, False), (12000, "cluster"),
                                   (32768, True), (32769, False), (40000, False)])
def test_bvh_keys_and_tree_bit_exact(n, dup):
    sc = _scene_n(n, dup=dup)
    rays = rays_from([0, 0, 3], [0, 0, -1], 1.0, 5.0, 0.01)
    dv = Dev(sc, rays).build()
    keys, children, bounds, scene_b = dv.bvh.export()
    torch.cuda.synchronize()
    ob, okeys = oracle.morton_keys(sc.t)
    np.testing.assert_array_equal(scene_b.cpu().numpy(), ob)
    sk = np.sort(okeys)
    np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64), sk)
    left, right = oracle.radix_tree(sk)
    ch = children.cpu().numpy()
    np.testing.assert_array_equal(ch[:, 0], left)
    np.testing.assert_array_equal(ch[:, 1], right)
    # boxes: every internal box contains its children; every leaf box contains the
    # corners of its primitive's oriented box (FP64)
    bb = bounds.cpu().numpy().astype(np.float64)
    for i in range(n - 1):
        for c in ch[i]:
            assert np.all(bb[i, :3] <= bb[c, :3]) and np.all(bb[i, 3:] >= bb[c, 3:])
    R = oracle.rotations(sc.q)
    corners = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float64)
    perm = (sk & np.uint64(0xFFFFFFFF)).astype(np.int64)
    for j in range(0, n, max(1, n // 500)):
        k = perm[j]
        pts = sc.t[k].astype(np.float64) + (corners * sc.s[k]) @ R[k].T
        leaf = bb[n - 1 + j]
        assert np.all(pts >= leaf[:3][None]) and np.all(pts <= leaf[3:][None])


def test_bvh_empty_and_rebuild_reuse():
    ctx = T.Context(0)
    sc0 = _scene_n(0)
    dv = Dev(sc0, rays_from([0, 0, 3], [0, 0, -1], 1.0, 5.0, 0.01), ctx=ctx).build()
    assert dv.bvh.size == 0
    # grow, shrink, grow again with one handle
    for n in (100, 10, 3000, 7):
        sc = _scene_n(n, seed=n)
        d2 = Dev(sc, dv.rays, ctx=ctx)
        d2.bvh = dv.bvh
        d2.build()
        keys, children, _, _ = dv.bvh.export()
        torch.cuda.synchronize()
        _, okeys = oracle.morton_keys(sc.t)
        np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64), np.sort(okeys))


# --------------------------------------------------------------------------- hit lists
def _hit_sets_equal(dv, rays, sc):
    offs, ids, tin, tout = dv.hitlists()
    offs, ids, tin, tout = offs.cpu().numpy(), ids.cpu().numpy(), tin.cpu().numpy(), tout.cpu().numpy()
    o_offs, o_ids, o_tin, o_tout, _ = oracle.hit_lists(sc.t, sc.q, sc.s, rays.o, rays.d, rays.t_near, rays.t_far,
                                                       "f32")
    np.testing.assert_array_equal(offs, o_offs)
    for r in range(rays.n):
        a, b = offs[r], offs[r + 1]
        order = np.argsort(ids[a:b], kind="stable")
        np.testing.assert_array_equal(ids[a:b][order], o_ids[a:b])
        np.testing.assert_array_equal(tin[a:b][order], o_tin[a:b].astype(np.float32))
        np.testing.assert_array_equal(tout[a:b][order], o_tout[a:b].astype(np.float32))
    return int(offs[-1])


@pytest.mark.parametrize("cfg", ["tiny_8x8^3_64x64", "small_512x8^3_96x128"])
def test_hitlists_bit_exact(cfg):
    sc, rays, _ = synthetic.make_config(cfg, 0)
    dv = Dev(sc, rays).build()
    H = _hit_sets_equal(dv, rays, sc)
    assert H > rays.n // 2


def test_hitlists_random_rays_1d_and_grazing():
    """Random ray origins/directions (1-D ray groups, ragged last group) plus rays
    aimed exactly at box corners and edges."""
    rng = np.random.default_rng(5)
    sc = synthetic.make_scene(300, 4, 3, layout="shell", s_range=(0.05, 0.2))
    n = 1000
    o = rng.normal(0, 3, (n, 3))
    target = sc.t[rng.integers(0, sc.n, n)].astype(np.float64)
    # aim half of the rays at a corner or an edge midpoint of a box
    R = oracle.rotations(sc.q)
    for i in range(0, n, 2):
        k = rng.integers(0, sc.n)
        y = rng.choice([-1.0, 1.0], 3)
        if i % 4 == 0:
            y[rng.integers(0, 3)] = 0.0
        target[i] = sc.t[k] + R[k] @ (y * sc.s[k])
    d = target - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = rays_from(o, d, 0.5, 9.0, 0.01)
    dv = Dev(sc, rays).build()
    _hit_sets_equal(dv, rays, sc)


# --------------------------------------------------------------------------- images
@pytest.mark.parametrize("cfg", ["tiny_8x8^3_64x64", "small_512x8^3_96x128", "small_4096x16^3_83x128"])
def test_forward_matches_oracle(cfg):
    sc, rays, _ = synthetic.make_config(cfg, 0)
    dv = Dev(sc, rays).build()
    out, _ = dv.render()
    ref = oracle.render(sc, rays, F32M)
    _check_image(out.cpu().numpy(), ref["rgba"], cfg)
    assert (ref["rgba"][:, 3] > 0).mean() > 0.2  # the image is not mostly empty


def test_forward_1d_rays_equal_2d_tiles():
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 1)
    dv = Dev(sc, rays).build()
    a, _ = dv.render()
    rays.width = rays.height = 0
    dv1 = Dev(sc, rays).build()
    b, _ = dv1.render()
    # the same per-ray arithmetic in a different tiling: identical up to summation order
    assert (a - b).abs().max().item() < 1e-5


@pytest.mark.parametrize("eps,bg", [(0.0, (0.3, 0.6, 0.9)), (0.05, (0.0, 0.0, 0.0)), (0.2, (1.0, 0.5, 0.0))])
def test_forward_eps_and_background(eps, bg):
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 2)
    rays.eps_early, rays.bg = eps, bg
    dv = Dev(sc, rays).build()
    out, _ = dv.render()
    ref = oracle.render(sc, rays, F32M)["rgba"]
    g = out.cpu().numpy()
    if eps == 0.0:
        _check_image(g, ref, f"bg{bg}")
    else:
        # the stop test T >= 1 - eps may land one sample apart (FP32 vs FP64); each
        # side is within eps of the eps = 0 image
        rays.eps_early = 0.0
        ref0 = oracle.render(sc, rays, F32M)["rgba"]
        assert np.abs(g - ref0).max() <= eps + 2e-4
        err = np.abs(g - ref).max(1)
        assert (err <= 2e-4).mean() >= 0.99


def test_forward_literal_composite():
    """MVP_COMPOSITE_LITERAL: A I + (1 - A) B, against the oracle's literal mode."""
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 2)
    rays.bg = (0.25, 0.5, 1.0)
    dv = Dev(sc, rays)
    dv.rs = T.rays_struct(dv.o, dv.d, literal_composite=True, **dv.params)
    out, _ = dv.build().render()
    ref = oracle.render(sc, rays, F32M | oracle.LITERAL)["rgba"]
    _check_image(out.cpu().numpy(), ref, "literal composite")
    pre = oracle.render(sc, rays, F32M)["rgba"]
    assert np.abs(ref - pre).max() > 1e-2
    g = torch.zeros_like(out)
    _, saved = T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, dv.rs, want_saved=True)
    with pytest.raises(B.MVPError) as ei:
        T.raymarch_bwd(dv.ctx, dv.prims, dv.bvh, dv.rs, saved, g)
    assert ei.value.status == B.MVP_ERR_INVALID_ARG


def test_forward_empty_scene_and_zero_payload():
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 0)
    rays.bg = (0.1, 0.2, 0.3)
    empty = synthetic.Scene(t=sc.t[:0], q=sc.q[:0], s=sc.s[:0], payload=sc.payload[:0], M=sc.M)
    dv = Dev(empty, rays).build()
    out, _ = dv.render()
    o = out.cpu().numpy()
    np.testing.assert_array_equal(o[:, :3], np.broadcast_to(np.float32(rays.bg), (rays.n, 3)))
    assert np.all(o[:, 3] == 0)
    zero = synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, payload=np.zeros_like(sc.payload), M=sc.M)
    dv = Dev(zero, rays).build()
    out, _ = dv.render()
    assert torch.all(out[:, 3] == 0)


def test_forward_uniform_box_closed_form():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "uniform_box.json")))
    b, r = g["box"], g["ray"]
    for case in g["cases"]:
        sc = single_box(M=b["M"], alpha=case["sigma"], rgb=b["rgb"], t=b["t"], q=b["q"], s=b["s"])
        rays = rays_from(r["o"], r["d"], r["t_near"], r["t_far"], r["dt"], eps=case["eps"])
        dv = Dev(sc, rays).build()
        out, _ = dv.render()
        o = out.cpu().numpy()[0]
        assert abs(o[3] - case["A"]) < 1e-5
        np.testing.assert_allclose(o[:3], case["I"], atol=1e-5)
        n = dv.count().cpu().numpy()[0]
        assert n == case["n_inside"]


def test_forward_saturation_hides_content_behind():
    front = single_box(M=3, alpha=50.0, rgb=(0.9, 0.1, 0.2), t=(0, 0, 0), s=(0.3, 0.3, 0.3))
    back_a = single_box(M=3, alpha=2.0, rgb=(0.1, 0.8, 0.3), t=(0, 0, 1.0), s=(0.3, 0.3, 0.3))
    back_b = single_box(M=3, alpha=7.0, rgb=(0.5, 0.5, 0.5), t=(0.05, 0, 1.2), s=(0.35, 0.3, 0.3))
    d = np.array([[0, 0, 1], [0.02, 0.01, 1]], np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = rays_from([0, 0, -3], d, 0.0, 8.0, 0.005)
    a, _ = Dev(concat_scenes(front, back_a), rays).build().render()
    b, _ = Dev(concat_scenes(front, back_b), rays).build().render()
    assert torch.all(a[:, 3] == 1.0)
    assert torch.equal(a, b)


def test_forward_permutation_invariance():
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 2)
    perm = np.random.default_rng(1).permutation(sc.n)
    from helpers import permute_scene
    a, _ = Dev(sc, rays).build().render()
    b, _ = Dev(permute_scene(sc, perm), rays).build().render()
    assert (a - b).abs().max().item() < 1e-5


def _stack_scene(n, seed):
    """n boxes of equal size stacked almost on top of each other (jittered centres,
    random rotations), low opacity: every ray through the middle meets all of them at
    the same samples."""
    rng = np.random.default_rng(seed)
    base = single_box(M=3, alpha=0.004, s=(0.5, 0.5, 0.5))
    payload = np.repeat(base.payload, n, 0)
    payload[..., :3] = rng.uniform(0.0, 1.0, (n, 1, 1, 1, 3)).astype(np.float32)
    payload[..., 3] *= rng.uniform(0.5, 1.5, (n, 3, 3, 3)).astype(np.float32)
    t = rng.uniform(-0.05, 0.05, (n, 3)).astype(np.float32)
    return synthetic.Scene(t=t, q=synthetic.random_unit_quaternions(rng, n), s=np.repeat(base.s, n, 0),
                           payload=payload, M=3)


@pytest.mark.parametrize("n", [48, 49, 80, 150])
def test_overlap_beyond_a_tile_window(n):
    """Up to and well beyond the 48 primitives a tile's window list holds meeting one
    sample: the tile sums all of them (no error), image and evaluation counts as the
    oracle's."""
    sc = _stack_scene(n, n)
    cam = synthetic.look_at_camera((0.3, -0.2, -3.0), 20, 12, 16.0)
    rays = synthetic.make_rays([cam], 1.0, 5.0, 0.02)
    dv = Dev(sc, rays).build()
    out, _ = dv.render()  # raises on a device status bit
    ref = oracle.render(sc, rays, F32M)
    _check_image(out.cpu().numpy(), ref["rgba"], f"stack{n}")
    cnt = dv.count().cpu().numpy()
    same = np.abs(out.cpu().numpy() - ref["rgba"]).max(1) < 2e-4
    np.testing.assert_array_equal(cnt[same], ref["n_eval"][same])
    assert ref["n_eval"].max() >= n  # some ray evaluates every box


@pytest.mark.parametrize("n", [49, 150])
def test_backward_overlap_beyond_a_tile_window(n):
    """The adjoint on the same scenes: gradients within 1e-3 of the oracle adjoint."""
    sc = _stack_scene(n, n + 1)
    cam = synthetic.look_at_camera((0.3, -0.2, -3.0), 20, 12, 16.0)
    rays = synthetic.make_rays([cam], 1.0, 5.0, 0.02)
    dv = Dev(sc, rays).build()
    out, saved = T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, dv.rs, want_saved=True)
    g = np.random.default_rng(n).standard_normal((rays.n, 4))
    gt = torch.from_numpy(g.astype(np.float32)).cuda()
    gp = torch.zeros(dv.payload.shape, dtype=torch.float32, device="cuda")
    g_t, g_q, g_s = torch.zeros_like(dv.t), torch.zeros_like(dv.q), torch.zeros_like(dv.s)
    T.raymarch_bwd(dv.ctx, dv.prims, dv.bvh, dv.rs, saved, gt, gp, g_t, g_q, g_s)
    dv.ctx.sync()
    R = oracle.backward(sc, rays, g.astype(np.float32).astype(np.float64), F32M)
    for key, val in (("g_payload", gp), ("g_t", g_t), ("g_q", g_q), ("g_s", g_s)):
        v = val.cpu().numpy().astype(np.float64)
        rel = np.abs(v - R[key]).max() / max(np.abs(R[key]).max(), 1e-30)
        assert rel <= 1e-3, (key, rel)


def test_invalid_arguments():
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 0)
    dv = Dev(sc, rays).build()
    other = Dev(synthetic.make_scene(9, 8, 1), rays, ctx=dv.ctx)
    with pytest.raises(B.MVPError) as ei:  # BVH built for another primitive set
        T.raymarch_fwd(dv.ctx, other.prims, dv.bvh, dv.rs)
    assert ei.value.status == B.MVP_ERR_INVALID_ARG
    bad = T.rays_struct(dv.o, dv.d, t_near=5.0, t_far=1.0, dt=0.01)
    with pytest.raises(B.MVPError):
        T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, bad)
    bad = T.rays_struct(dv.o, dv.d, t_near=0.0, t_far=1000.0, dt=0.001)  # > 65535 samples
    with pytest.raises(B.MVPError):
        T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, bad)


# --------------------------------------------------------------------------- work counts
def test_eval_counts_match_oracle():
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 0)
    dv = Dev(sc, rays).build()
    n = dv.count().cpu().numpy()
    ref = oracle.render(sc, rays, F32M)["n_eval"]
    same = n == ref
    assert same.mean() >= 0.999, same.mean()
    assert np.abs(n - ref).max() <= 16


# --------------------------------------------------------------------------- cameras
def test_camera_rays_match_generator():
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 0)
    cam = rays.cameras[0]
    ctx = T.Context(0)
    o, d = T.camera_rays(ctx, cam.matrix34(), cam.focal, cam.width, cam.height)
    torch.cuda.synchronize()
    np.testing.assert_allclose(o.cpu().numpy(), rays.o, atol=1e-6)
    np.testing.assert_allclose(d.cpu().numpy(), rays.d, atol=2e-6)


# --------------------------------------------------------------------------- paper scale
@pytest.mark.parametrize("cfg", ["paper_4096x16^3_667x1024", "sweep_32768x8^3_667x1024", "sweep_512x32^3_667x1024"])
def test_paper_scale_sampled_pixels(cfg):
    """Full-size frame in the benchmark's launch configuration; 3000 seeded pixels
    are re-rendered by the oracle one by one."""
    sc, rays, _ = synthetic.make_config(cfg, 0)
    dv = Dev(sc, rays).build()
    out, _ = dv.render()
    o = out.cpu().numpy()
    sel = np.random.default_rng(0).choice(rays.n, 3000, replace=False)
    sub = rays_from(rays.o[sel], rays.d[sel], rays.t_near, rays.t_far, rays.dt)
    ref = oracle.render(sc, sub, F32M)["rgba"]
    _check_image(o[sel], ref, cfg)
    assert (ref[:, 3] > 0).mean() > 0.3


def test_degenerate_poses_reported():
    """A NaN centre, a zero quaternion and a negative scale are reported by the next
    sync (MVP_ERR_INVALID_ARG) and refused by avatar registration; those primitives are
    absent: the frame equals the oracle's image of the scene without them."""
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 4)
    bad = sc.t.copy(), sc.q.copy(), sc.s.copy()
    bad[0][5, 1] = np.nan
    bad[1][17] = 0.0
    bad[2][40, 2] = -sc.s[40, 2]
    sc_bad = synthetic.Scene(t=bad[0], q=bad[1], s=bad[2], payload=sc.payload, M=sc.M)
    dv = Dev(sc_bad, rays)
    dv.bvh.build(dv.prims)
    with pytest.raises(B.MVPError) as ei:
        dv.ctx.sync()
    assert ei.value.status == B.MVP_ERR_INVALID_ARG
    out, _ = T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, dv.rs)
    dv.ctx.sync()  # the status word was cleared; the render itself reports nothing
    keep = np.setdiff1d(np.arange(sc.n), [5, 17, 40])
    ok = synthetic.Scene(t=sc.t[keep], q=sc.q[keep], s=sc.s[keep], payload=sc.payload[keep], M=sc.M)
    ref = oracle.render(ok, rays, F32M)["rgba"]
    _check_image(out.cpu().numpy(), ref, "degenerate poses")
    # the bad primitives were in view: the image without them differs from the full one
    full = oracle.render(sc, rays, F32M)["rgba"]
    assert np.abs(full - ref).max() > 1e-2
    srv = T.Server(dv.ctx, hbm_budget=1 << 30, max_slots=2)
    with pytest.raises(B.MVPError) as ei:
        srv.register(dv.t, dv.q, dv.s, dv.payload)
    assert ei.value.status == B.MVP_ERR_INVALID_ARG
    assert srv.register(*(torch.from_numpy(x).cuda() for x in (sc.t, sc.q, sc.s, sc.payload))) == 0
    srv.close()


def test_tile_schedule_changes_no_result():
    """The frame kernel's cost-ordered tile schedule (heaviest tiles of the last frame
    first) and the plain order give the same image bit for bit, on one stream and when
    calls alternate between two streams."""
    sc, rays, _ = synthetic.make_config("small_4096x16^3_83x128", 1)
    dv = Dev(sc, rays).build()
    dv.ctx.set_tile_schedule(False)
    plain, _ = dv.render()
    dv.ctx.set_tile_schedule(True)
    for _ in range(3):  # the first frame records costs, the next ones use them
        out, _ = dv.render()
        assert torch.equal(out, plain)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for k in range(6):
        with torch.cuda.stream(s1 if k % 2 else s2):
            o, _ = T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, dv.rs)
            outs.append(o)
    torch.cuda.synchronize()
    dv.ctx.sync()
    for o in outs:
        assert torch.equal(o, plain)
    ref = oracle.render(sc, rays, F32M)["rgba"]
    _check_image(plain.cpu().numpy(), ref, "tile schedule")


def test_largest_sample_count_and_voxel_edge():
    """The limits of the boundary: n_steps = MVP_MAX_STEPS (65535 samples; the primitives'
    sample spans exceed what a window's 8-bit lane offsets hold, so windows split) and payload
    edge M = MVP_MAX_M (128)."""
    sc = synthetic.make_scene(8, 8, 3, layout="sphere", s_const=0.3, empty_frac=0.5)
    cam = synthetic.look_at_camera((0.0, 0.0, -3.0), 24, 20, 24.0)
    rays = synthetic.make_rays([cam], 0.0, 6.55345, 1e-4)
    assert rays.n_steps == 65535 == B.lib().mvp_num_steps(0.0, 6.55345, 1e-4)
    out, _ = Dev(sc, rays).build().render()
    ref = oracle.render(sc, rays, F32M)
    _check_image(out.cpu().numpy(), ref["rgba"], "65535 samples")
    assert ref["i_last"].max() == 65534 and (ref["rgba"][:, 3] > 0).mean() > 0.3
    big = synthetic.make_scene(2, 128, 4, layout="sphere", s_const=0.6, empty_frac=0.3)
    cam = synthetic.look_at_camera((0.2, 0.1, -3.0), 40, 32, 40.0)
    rays = synthetic.make_rays([cam], 1.0, 5.0, 0.005)
    out, _ = Dev(big, rays).build().render()
    ref = oracle.render(big, rays, F32M)
    _check_image(out.cpu().numpy(), ref["rgba"], "M = 128")
    assert (ref["rgba"][:, 3] > 0).mean() > 0.3


def test_frame_replays_as_a_cuda_graph():
    """With the tile schedule off the frame (BVH rebuild + march) enqueues kernels only,
    so it can be captured into a CUDA graph; replays give the eager image bit for bit."""
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 2)
    dv = Dev(sc, rays).build()
    dv.ctx.set_tile_schedule(False)
    eager, _ = dv.render()
    out = torch.empty_like(eager)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up on the capture stream (no allocation inside the capture)
        dv.bvh.build(dv.prims)
        T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, dv.rs, out=out)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        dv.bvh.build(dv.prims)
        T.raymarch_fwd(dv.ctx, dv.prims, dv.bvh, dv.rs, out=out)
    for _ in range(3):
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)
    dv.ctx.sync()
