"""Serving (continuous batching: one launch per admitted request, requests overlapping on the GPU).

Each request's image must equal mvp_camera_rays + mvp_raymarch_fwd on the same
avatar, and must be the same whether the request runs alone or in a mix of many
concurrent requests of other avatars, cameras and resolutions. Every served image
(alone, in the mix, each eye of a binocular request) also meets the FP64 oracle at
the definition bar. Admission honours the HBM budget; oversize requests are refused;
waits time out on the host.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from helpers import rays_from_matrix
from parity_rules import definition_bar

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from gpu_util import DEV  # noqa: E402
from paper_2103_01954_gb300 import binding as B  # noqa: E402
from paper_2103_01954_gb300 import torch_ops as T  # noqa: E402

T_NEAR, T_FAR, DT = 1.0, 5.0, 0.01
F64M = oracle.MODE_PRUNED | oracle.MEMBER_F64
SPECS = [(256, 8, torch.float32, 0), (1024, 6, torch.bfloat16, 1), (64, 16, torch.float16, 2)]


def _scene(n, M, seed):
    return synthetic.make_scene(n, M, seed, layout="shell", s_range=(0.04 * (4096 / n) ** 0.5, 0.08 * (4096 / n) ** 0.5))


def _avatars(ctx):
    """Three small avatars of different sizes and payload types (FP32, BF16, FP16)."""
    out = []
    for n, M, dt, seed in SPECS:
        sc = _scene(n, M, seed)
        t = torch.from_numpy(sc.t).to(DEV)
        q = torch.from_numpy(sc.q).to(DEV)
        s = torch.from_numpy(sc.s).to(DEV)
        p32 = torch.from_numpy(sc.payload).to(DEV)
        p = p32 if dt == torch.float32 else T.pack_payload(ctx, p32, dt)
        out.append((t, q, s, p))
    return out


def _oracle_scenes():
    """The avatars as the oracle sees them: BF16 / FP16 payloads dequantised (the exact
    values the kernel reads)."""
    out = []
    for n, M, dt, seed in SPECS:
        sc = _scene(n, M, seed)
        if dt != torch.float32:
            sc = synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, M=sc.M,
                                 payload=torch.from_numpy(sc.payload).to(dt).float().numpy())
        out.append(sc)
    return out


def _oracle_image(sc, cam, w, h):
    rays = rays_from_matrix(cam, float(w), w, h, T_NEAR, T_FAR, DT)
    return oracle.render(sc, rays, F64M)


def _reference(ctx, av, cam, focal, w, h):
    t, q, s, p = av
    prims = T.prims_struct(t, q, s, p)
    bvh = T.BVH(ctx)
    bvh.build(prims)
    o, d = T.camera_rays(ctx, cam, focal, w, h)
    rs = T.rays_struct(o, d, t_near=T_NEAR, t_far=T_FAR, dt=DT, width=w, height=h)
    out, _ = T.raymarch_fwd(ctx, prims, bvh, rs)
    ctx.sync()
    return out


def _cams(n, seed):
    rng = np.random.default_rng(seed)
    return [synthetic.random_camera(rng, 3.0, 1, 1, 1.0).matrix34() for _ in range(n)]


def test_serving_matches_single_render_and_mix():
    torch.cuda.set_device(0)
    ctx = T.Context(0)
    avs = _avatars(ctx)
    srv = T.Server(ctx, hbm_budget=2 << 30, max_slots=16)
    ids = [srv.register(*a) for a in avs]
    sizes = [(64, 48), (96, 96), (33, 70), (128, 64)]
    cams = _cams(12, 3)
    reqs = [(ids[i % 3], cams[i], sizes[i % 4]) for i in range(12)]
    # alone: one request at a time
    alone = []
    for aid, cam, (w, h) in reqs:
        tk = srv.submit_raw(T.Server.request(aid, cam, float(w), w, h, T_NEAR, T_FAR, DT))
        out = torch.empty((h * w, 4), dtype=torch.float32, device=DEV)
        st, _ = srv.wait(tk, 10000.0, out)
        assert st == B.MVP_OK
        alone.append(out)
    # in the mix: all submitted back to back, polled out of order
    tks = [srv.submit_raw(T.Server.request(aid, cam, float(w), w, h, T_NEAR, T_FAR, DT)) for aid, cam, (w, h) in reqs]
    mix = [torch.empty((h * w, 4), dtype=torch.float32, device=DEV) for _, _, (w, h) in reqs]
    for j in reversed(range(len(tks))):
        st, _ = srv.wait(tks[j], 10000.0, mix[j])
        assert st == B.MVP_OK
    stats = srv.stats()
    assert stats["device_status"] == 0
    assert stats["max_in_flight"] >= 4  # the burst was in flight together
    for (aid, cam, (w, h)), a, m in zip(reqs, alone, mix):
        assert torch.equal(a, m), "alone and in the mix differ"
        ref = _reference(ctx, avs[aid], cam, float(w), w, h)
        assert (a - ref).abs().max().item() <= 1e-5
        assert a[:, 3].max().item() > 0  # the avatar is in view
    srv.close()


def test_admission_respects_budget_and_frees_memory():
    torch.cuda.set_device(0)
    ctx = T.Context(0)
    av = _avatars(ctx)[0]
    probe = T.Server(ctx, hbm_budget=1 << 30)
    probe.register(*av)
    resident = probe.stats()["resident_bytes"]
    probe.close()
    w = h = 64
    img = w * h * 16
    srv = T.Server(ctx, hbm_budget=resident + 2 * img + 100, max_slots=8)
    aid = srv.register(*av)
    cams = _cams(6, 7)
    tks = [srv.submit_raw(T.Server.request(aid, c, 64.0, w, h, T_NEAR, T_FAR, DT)) for c in cams]
    st = srv.stats()
    assert st["in_flight"] <= 2 and st["pending"] >= 4
    outs = []
    for tk in tks:
        out = torch.empty((h * w, 4), dtype=torch.float32, device=DEV)
        s_, _ = srv.wait(tk, 10000.0, out)
        assert s_ == B.MVP_OK
        outs.append(out)
    st = srv.stats()
    assert st["max_in_flight"] <= 2 and st["completed"] == 6 and st["in_flight_bytes"] == 0
    for c, o in zip(cams, outs):
        assert (o - _reference(ctx, av, c, 64.0, w, h)).abs().max().item() <= 1e-5
    # a request whose image alone exceeds the budget is refused
    with pytest.raises(B.MVPError) as ei:
        srv.submit_raw(T.Server.request(aid, cams[0], 64.0, 512, 512, T_NEAR, T_FAR, DT))
    assert ei.value.status == B.MVP_ERR_CAPACITY
    srv.close()


def test_wait_timeout_unknown_ticket_and_bad_avatar():
    torch.cuda.set_device(0)
    ctx = T.Context(0)
    av = _avatars(ctx)[0]
    probe = T.Server(ctx, hbm_budget=1 << 30)
    probe.register(*av)
    resident = probe.stats()["resident_bytes"]
    probe.close()
    w = h = 32
    srv = T.Server(ctx, hbm_budget=resident + w * h * 16 + 100, max_slots=4)
    aid = srv.register(*av)
    cams = _cams(2, 9)
    t1 = srv.submit_raw(T.Server.request(aid, cams[0], 32.0, w, h, T_NEAR, T_FAR, DT))
    t2 = srv.submit_raw(T.Server.request(aid, cams[1], 32.0, w, h, T_NEAR, T_FAR, DT))
    # t2 cannot be admitted until t1 is collected: a wait on it runs out
    st, _ = srv.wait(t2, 5.0)
    assert st == B.MVP_ERR_TIMEOUT
    st, _ = srv.wait(t1, 10000.0)
    assert st == B.MVP_OK
    st, _ = srv.wait(t2, 10000.0)
    assert st == B.MVP_OK
    with pytest.raises(B.MVPError):
        srv.poll(12345)
    with pytest.raises(B.MVPError) as ei:
        srv.submit_raw(T.Server.request(7, cams[0], 32.0, w, h, T_NEAR, T_FAR, DT))
    assert ei.value.status == B.MVP_ERR_INVALID_ARG
    srv.close()


def test_stereo_request_equals_two_mono_requests():
    """A binocular request (two cameras, one launch, the avatar's one BVH) gives, per
    eye, the image of the corresponding mono request, bit for bit."""
    torch.cuda.set_device(0)
    ctx = T.Context(0)
    avs = _avatars(ctx)
    srv = T.Server(ctx, hbm_budget=2 << 30, max_slots=8)
    ids = [srv.register(*a) for a in avs]
    w, h = 72, 56  # ragged tiles in both directions
    cam = _cams(1, 11)[0]
    right = cam.copy()
    right[:, 3] += 0.064 * right[:, 0]  # eye moved 6.4 cm along the camera's right axis
    for aid, av in zip(ids, avs):
        tk = srv.submit_raw(T.Server.request(aid, cam, float(w), w, h, T_NEAR, T_FAR, DT, c2w_right=right))
        both = torch.empty((2, h * w, 4), dtype=torch.float32, device=DEV)
        st, _ = srv.wait(tk, 10000.0, both)
        assert st == B.MVP_OK
        for eye, c in ((0, cam), (1, right)):
            tk = srv.submit_raw(T.Server.request(aid, c, float(w), w, h, T_NEAR, T_FAR, DT))
            mono = torch.empty((h * w, 4), dtype=torch.float32, device=DEV)
            st, _ = srv.wait(tk, 10000.0, mono)
            assert st == B.MVP_OK
            assert torch.equal(both[eye], mono)
            ref = _reference(ctx, av, c, float(w), w, h)
            assert (mono - ref).abs().max().item() <= 1e-5
        assert not torch.equal(both[0], both[1])  # the eyes see different images
    assert srv.stats()["device_status"] == 0
    srv.close()


def test_request_payload_override():
    """A request carrying its own (view-dependent) payload renders exactly what an avatar
    registered with that payload renders, mono and stereo; a misaligned one is refused."""
    torch.cuda.set_device(0)
    ctx = T.Context(0)
    av = _avatars(ctx)[1]  # BF16
    t, q, s, p = av
    n, M = p.shape[0], p.shape[1]
    rgb = torch.rand((n, M, M, M, 3), device=DEV)
    op = p[..., 3].float().contiguous()
    pv = T.assemble_payload(ctx, rgb, op, torch.bfloat16, 0.0, 8)  # same opacity, another view's colour
    ctx.sync()
    srv = T.Server(ctx, hbm_budget=2 << 30, max_slots=8)
    a_base = srv.register(t, q, s, p)
    a_view = srv.register(t, q, s, pv)
    w, h = 72, 56
    cam = _cams(1, 5)[0]
    right = cam.copy()
    right[:, 3] += 0.064 * right[:, 0]
    for c2 in (None, right):
        nv = 1 if c2 is None else 2
        imgs = []
        for aid, payload in ((a_base, pv), (a_view, None), (a_base, None)):
            tk = srv.submit_raw(T.Server.request(aid, cam, float(w), w, h, T_NEAR, T_FAR, DT, c2w_right=c2,
                                                 payload=payload))
            img = torch.empty((nv, h * w, 4), dtype=torch.float32, device=DEV)
            st, _ = srv.wait(tk, 10000.0, img)
            assert st == B.MVP_OK
            imgs.append(img)
        assert torch.equal(imgs[0], imgs[1])      # override == avatar registered with it
        assert not torch.equal(imgs[0], imgs[2])  # and not the avatar's own payload
    bad = T.Server.request(a_base, cam, float(w), w, h, T_NEAR, T_FAR, DT)
    bad.payload = pv.data_ptr() + 4
    with pytest.raises(B.MVPError) as ei:
        srv.submit_raw(bad)
    assert ei.value.status == B.MVP_ERR_INVALID_ARG
    assert srv.stats()["device_status"] == 0
    srv.close()


def test_cancel_queued_and_running_requests():
    """A queued request is dropped before it runs; a running one finishes and is freed
    by the server; both tickets become unknown; the others complete unchanged."""
    torch.cuda.set_device(0)
    ctx = T.Context(0)
    av = _avatars(ctx)[0]
    srv = T.Server(ctx, hbm_budget=2 << 30, max_slots=2)
    aid = srv.register(*av)
    w, h = 200, 160
    cams = _cams(6, 21)
    tks = [srv.submit_raw(T.Server.request(aid, c, float(w), w, h, T_NEAR, T_FAR, DT)) for c in cams]
    st = srv.stats()
    assert st["in_flight"] + st["pending"] == 6 and st["pending"] >= 4  # two slots
    srv.cancel(tks[4])  # queued
    srv.cancel(tks[0])  # admitted (running or done)
    for tk in (tks[0], tks[4]):
        with pytest.raises(B.MVPError) as ei:
            srv.poll(tk)
        assert ei.value.status == B.MVP_ERR_INVALID_ARG
        with pytest.raises(B.MVPError):
            srv.cancel(tk)
    for i in (1, 2, 3, 5):
        img = torch.empty((h * w, 4), dtype=torch.float32, device=DEV)
        st, _ = srv.wait(tks[i], 10000.0, img)
        assert st == B.MVP_OK
        assert (img - _reference(ctx, av, cams[i], float(w), w, h)).abs().max().item() <= 1e-5
    st = srv.stats()
    assert st["cancelled"] == 2 and st["completed"] == 4
    assert st["pending"] == 0 and st["in_flight"] == 0 and st["in_flight_bytes"] == 0
    assert st["device_status"] == 0
    srv.close()


def test_served_images_match_the_oracle():
    """Every served image against the FP64 oracle at the definition bar: requests of three
    avatars (FP32, BF16, FP16 payloads) at several resolutions, rendered alone, then all
    at once in a mix, and binocular requests (each eye). The oracle's rays come from the
    request's own camera matrix through an FP64 pinhole model."""
    torch.cuda.set_device(0)
    ctx = T.Context(0)
    avs = _avatars(ctx)
    scenes = _oracle_scenes()
    srv = T.Server(ctx, hbm_budget=2 << 30, max_slots=16)
    ids = [srv.register(*a) for a in avs]
    sizes = [(64, 48), (96, 96), (33, 70), (128, 64)]
    cams = _cams(9, 31)
    reqs = [(i % 3, cams[i], sizes[i % 4]) for i in range(9)]

    def submit(k, cam, w, h, right=None):
        return srv.submit_raw(T.Server.request(ids[k], cam, float(w), w, h, T_NEAR, T_FAR, DT, c2w_right=right))

    alone = []
    for k, cam, (w, h) in reqs:
        out = torch.empty((h * w, 4), dtype=torch.float32, device=DEV)
        st, _ = srv.wait(submit(k, cam, w, h), 10000.0, out)
        assert st == B.MVP_OK
        alone.append(out.cpu().numpy())
    tks = [submit(k, cam, w, h) for k, cam, (w, h) in reqs]
    mix = [torch.empty((h * w, 4), dtype=torch.float32, device=DEV) for _, _, (w, h) in reqs]
    for j in reversed(range(len(tks))):
        st, _ = srv.wait(tks[j], 10000.0, mix[j])
        assert st == B.MVP_OK
    assert srv.stats()["max_in_flight"] >= 4
    for (k, cam, (w, h)), a, m in zip(reqs, alone, mix):
        ref = _oracle_image(scenes[k], cam, w, h)
        label = f"served avatar {k} {w}x{h}"
        definition_bar(a, ref, label + " alone")
        definition_bar(m.cpu().numpy(), ref, label + " in the mix")
        assert (ref["rgba"][:, 3] > 0).mean() > 0.05
    # binocular requests: each eye against the oracle's image of that eye's camera
    w, h = 72, 56
    for k in range(3):
        cam = cams[k]
        right = cam.copy()
        right[:, 3] += np.float32(0.064) * right[:, 0]
        both = torch.empty((2, h * w, 4), dtype=torch.float32, device=DEV)
        st, _ = srv.wait(submit(k, cam, w, h, right), 10000.0, both)
        assert st == B.MVP_OK
        for eye, c in ((0, cam), (1, right)):
            definition_bar(both[eye].cpu().numpy(), _oracle_image(scenes[k], c, w, h), f"stereo avatar {k} eye {eye}")
    assert srv.stats()["device_status"] == 0
    srv.close()
