"""A fixed GPU workload over every kernel family of the library (BVH build at both
sizes, forward with window splitting and the list-free overflow path, sequential
blending, evaluation counts, hit lists, adjoint, serving with a stereo request, the
allocation-free entry point, decode-side epilogues), run once with the release
library and once, in a child process, with the checked build (MVP_CHECK_BOUNDS=1),
whose device-side bounds checks must stay silent and whose results must match.

Run as a script: ``python tests/checked_workload.py OUT.npz`` writes the results.
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _stack(n, seed, M=3):
    import synthetic

    rng = np.random.default_rng(seed)
    payload = np.zeros((n, M, M, M, 4), np.float32)
    payload[..., :3] = rng.uniform(0.0, 1.0, (n, 1, 1, 1, 3)).astype(np.float32)
    payload[..., 3] = 0.004 * rng.uniform(0.5, 1.5, (n, M, M, M)).astype(np.float32)
    t = rng.uniform(-0.05, 0.05, (n, 3)).astype(np.float32)
    return synthetic.Scene(t=t, q=synthetic.random_unit_quaternions(rng, n), s=np.full((n, 3), 0.5, np.float32),
                           payload=payload, M=M)


def run() -> dict:
    import torch

    import synthetic
    from paper_2103_01954_gb300 import binding as B
    from paper_2103_01954_gb300 import torch_ops as T

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    ctx = T.Context(0)
    res = {"checked": np.array([B.lib().mvp_bounds_checked()])}

    def up(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    def frame(name, sc, rays, dtype=torch.float32, sequential=False, grads=False):
        t, q, s = up(sc.t), up(sc.q), up(sc.s)
        p = up(sc.payload)
        if dtype != torch.float32:
            p = T.pack_payload(ctx, p, dtype)
        o, d = up(rays.o), up(rays.d)
        prims = T.prims_struct(t, q, s, p)
        rs = T.rays_struct(o, d, t_near=rays.t_near, t_far=rays.t_far, dt=rays.dt, eps_early=rays.eps_early,
                           bg=tuple(rays.bg), width=rays.width, height=rays.height, sequential=sequential)
        bvh = T.BVH(ctx)
        bvh.build(prims)
        out, saved = T.raymarch_fwd(ctx, prims, bvh, rs, want_saved=grads)
        cnt = T.raymarch_count(ctx, prims, bvh, rs)
        ctx.sync()
        res[name + "/rgba"] = out.cpu().numpy()
        res[name + "/count"] = cnt.cpu().numpy()
        if grads:
            g = torch.from_numpy(np.random.default_rng(7).standard_normal((rays.n, 4)).astype(np.float32)).to(dev)
            gp = torch.zeros(p.shape, dtype=torch.float32, device=dev)
            gt, gq, gs = torch.zeros_like(t), torch.zeros_like(q), torch.zeros_like(s)
            T.raymarch_bwd(ctx, prims, bvh, rs, saved, g, gp, gt, gq, gs)
            ctx.sync()
            for k, v in (("g_payload", gp), ("g_t", gt), ("g_q", gq), ("g_s", gs)):
                res[f"{name}/{k}"] = v.cpu().numpy()
        if not sequential:
            offs, ids, tin, tout = T.hitlists(ctx, prims, bvh, rs)
            ctx.sync()
            res[name + "/hit_offs"] = offs.cpu().numpy()
            res[name + "/hit_ids"] = ids.cpu().numpy()
        if rays.n and sc.n <= 16384:
            st = torch.full((1,), -1, dtype=torch.int32, device=dev)
            so = torch.empty_like(out)
            B.check(B.lib().mvp_raymarch_fwd_static(ctypes.byref(prims), ctypes.byref(rs),
                                                    ctypes.c_void_p(so.data_ptr()), ctypes.c_void_p(st.data_ptr()),
                                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
                    "mvp_raymarch_fwd_static")
            torch.cuda.synchronize()
            res[name + "/static"] = so.cpu().numpy()
            res[name + "/static_status"] = st.cpu().numpy()

    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 0)
    frame("tiny", sc, rays, grads=True)
    sc, rays, _ = synthetic.make_config("small_4096x16^3_83x128", 0)
    frame("small4096", sc, rays)
    frame("small4096_bf16", sc, rays, dtype=torch.bfloat16)
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 1)
    frame("small512_seq", sc, rays, sequential=True)
    sc = synthetic.make_scene(9000, 4, 2, layout="shell", s_range=(0.02, 0.05))  # the multi-launch BVH build
    cam = synthetic.look_at_camera((0.2, -0.1, -3.0), 48, 40, 48.0)
    frame("n9000", sc, synthetic.make_rays([cam], 1.0, 5.0, 0.01))
    cam = synthetic.look_at_camera((0.3, -0.2, -3.0), 20, 12, 16.0)
    rays = synthetic.make_rays([cam], 1.0, 5.0, 0.02)
    frame("stack150", _stack(150, 3), rays, grads=True)  # window splitting and the overflow path
    frame("stack150_m8", _stack(150, 4, M=8), rays)  # the same with 64-entry windows (8^3 payloads)
    # the adjoint replayed primitive group by primitive group (mask, work list, persistent replay)
    ctx.set_bwd_group_bytes(1)
    frame("stack150_grouped", _stack(150, 3), rays, grads=True)
    sc, rays_s, _ = synthetic.make_config("small_512x8^3_96x128", 1)
    frame("small512_seq_grouped", sc, rays_s, sequential=True, grads=True)
    ctx.set_bwd_group_bytes(0)
    # decode-side epilogues
    rng = np.random.default_rng(5)
    rgb = up(rng.uniform(0, 1, (64, 8, 8, 8, 3)).astype(np.float32))
    op = up(rng.uniform(0, 4, (64, 8, 8, 8)).astype(np.float32))
    res["assemble"] = T.assemble_payload(ctx, rgb, op, torch.bfloat16).float().cpu().numpy()
    # serving: a stereo request and a mono one of another avatar
    srv = T.Server(ctx, hbm_budget=1 << 30, max_slots=4)
    scs = [synthetic.make_scene(256, 8, 0), synthetic.make_scene(1024, 6, 1)]
    ids = [srv.register(up(s.t), up(s.q), up(s.s), up(s.payload)) for s in scs]
    c2w = synthetic.random_camera(np.random.default_rng(11), 3.0, 1, 1, 1.0).matrix34()
    right = c2w.copy()
    right[:, 3] += 0.064 * right[:, 0]
    for i, aid in enumerate(ids):
        w, h = 72, 56
        img = torch.empty((2, h * w, 4), dtype=torch.float32, device=dev)
        tk = srv.submit_raw(T.Server.request(aid, c2w, float(w), w, h, 1.0, 5.0, 0.01, c2w_right=right))
        st, _ = srv.wait(tk, 10000.0, img)
        B.check(st, "serve wait")
        res[f"serve{i}"] = img.cpu().numpy()
    res["serve_status"] = np.array([srv.stats()["device_status"]])
    srv.close()
    ctx.sync()
    return res


if __name__ == "__main__":
    out = run()
    np.savez(sys.argv[1], **out)
    print("ok", len(out))
