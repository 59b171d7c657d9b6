"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these compare the oracle with itself: each expected value comes from a
closed form, a library routine (scipy rotations, torch grid_sample), an invariance,
brute force, or a hand-derived golden fixture.
"""
import json
import os

import numpy as np
import pytest
import torch

import synthetic
from helpers import (concat_scenes, permute_scene, quat_from_matrix, rays_from, rot_matrix,
                     single_box)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

BRUTE64 = 0
PRUNED64 = 1
BRUTE32 = 2
PRUNED32 = 3
ALL_MODES = [BRUTE64, PRUNED64, BRUTE32, PRUNED32]


# --------------------------------------------------------------------------- Sec. 3.1.2
def test_rotation_matches_scipy(orc):
    rng = np.random.default_rng(1)
    q = rng.standard_normal((64, 4)).astype(np.float32) * 3.0  # unnormalised on purpose
    R = orc.rotations(q)
    np.testing.assert_allclose(R, rot_matrix(q), atol=1e-12)
    R32 = orc.rotations_f32spec(q)
    np.testing.assert_allclose(R32, R, atol=2e-6)
    np.testing.assert_allclose(np.einsum("kij,kil->kjl", R, R), np.broadcast_to(np.eye(3), R.shape),
                               atol=1e-12)


# --------------------------------------------------------------------------- Sec. 3.2.2 golden
@pytest.mark.parametrize("mode", ALL_MODES)
def test_uniform_box_golden(orc, mode):
    g = json.load(open(os.path.join(GOLDEN, "uniform_box.json")))
    b, r = g["box"], g["ray"]
    for case in g["cases"]:
        sc = single_box(M=b["M"], alpha=case["sigma"], rgb=b["rgb"], t=b["t"], q=b["q"], s=b["s"])
        rays = rays_from(r["o"], r["d"], r["t_near"], r["t_far"], r["dt"], eps=case["eps"])
        assert rays.n_steps == r["n_steps"]
        out = orc.render(sc, rays, mode)
        tol = g["tolerance"]
        assert abs(out["rgba"][0, 3] - case["A"]) < tol
        np.testing.assert_allclose(out["rgba"][0, :3], case["I"], atol=tol)
        assert out["n_eval"][0] == case["n_inside"]
        assert out["i_clamp"][0] == case["i_clamp"]
        assert out["i_last"][0] == case["i_last"]


def test_uniform_box_continuum_limit(orc):
    """T -> min(sigma * L, 1) as dt -> 0 (L = chord length), within sigma*dt."""
    h, sigma = 0.3, 1.2
    sc = single_box(M=3, alpha=sigma, s=(h, h, h))
    for dt in (0.01, 0.002, 0.0005):
        rays = rays_from([0, 0, -3], [0, 0, 1], 0.0, 6.0, dt)
        A = orc.render(sc, rays, PRUNED64)["rgba"][0, 3]
        assert abs(A - min(sigma * 2 * h, 1.0)) <= sigma * dt + 1e-12


# --------------------------------------------------------------------------- Sec. 3.2.1 trilinear
@pytest.mark.parametrize("mode", [BRUTE64, PRUNED32])
def test_trilinear_matches_grid_sample(orc, mode):
    """One sample per ray inside one rotated box: its RGBA equals
    torch grid_sample(align_corners=True) of the payload at the local coordinates
    (a single primitive spanning the volume is the Neural Volumes setting, Sec. 4.3)."""
    rng = np.random.default_rng(7)
    M = 5
    q = synthetic.random_unit_quaternions(rng, 1)
    sc = synthetic.Scene(t=np.array([[0.3, -0.2, 0.1]], np.float32), q=q,
                         s=np.array([[0.5, 0.7, 0.9]], np.float32),
                         payload=rng.random((1, M, M, M, 4)).astype(np.float32), M=M)
    n = 200
    y = rng.uniform(-0.95, 0.95, (n, 3))
    R = rot_matrix(q[0])
    x = sc.t[0].astype(np.float64) + (R @ (y * sc.s[0]).T).T
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t0, dt = 2.0, 1e-3
    o = (x - t0 * d).astype(np.float32)
    d = d.astype(np.float32)
    rays = rays_from(o, d, t0, t0 + 0.5 * dt, dt)
    assert rays.n_steps == 1
    out = orc.render(sc, rays, mode)["rgba"]
    # the actual sample position from the float32 ray
    xs = o.astype(np.float64) + np.float64(np.float32(t0)) * d.astype(np.float64)
    ys = ((xs - sc.t[0].astype(np.float64)) @ R) / sc.s[0].astype(np.float64)
    inp = torch.from_numpy(sc.payload[0].astype(np.float64)).permute(3, 0, 1, 2)[None]
    grid = torch.from_numpy(ys)[None, None, None]  # (x, y, z) -> (W, H, D)
    ref = torch.nn.functional.grid_sample(inp, grid, mode="bilinear", align_corners=True)[0, :, 0, 0].T
    ref = ref.numpy()
    dt64 = float(np.float32(dt))
    alpha = out[:, 3] / dt64
    np.testing.assert_allclose(alpha, ref[:, 3], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(out[:, :3] / out[:, 3:4], ref[:, :3], rtol=1e-8, atol=1e-9)


def test_affine_field_exact(orc):
    """Trilinear interpolation reproduces an affine field exactly, so the march of a
    field alpha = a0 + a . (ix, iy, iz) has a closed-form sum. Distinct coefficients per
    axis catch a transposed payload layout (x must be the fastest axis)."""
    M = 6
    a0, a = 0.3, np.array([0.05, 0.11, 0.23])
    iz, iy, ix = np.meshgrid(np.arange(M), np.arange(M), np.arange(M), indexing="ij")
    payload = np.zeros((1, M, M, M, 4), np.float32)
    payload[0, ..., 3] = a0 + a[0] * ix + a[1] * iy + a[2] * iz
    payload[0, ..., 0] = 0.5
    payload[0, ..., 1] = 0.1 * ix
    payload[0, ..., 2] = 0.1 * iz
    s = np.array([0.4, 0.5, 0.6])
    sc = synthetic.Scene(t=np.zeros((1, 3), np.float32), q=np.array([[1, 0, 0, 0]], np.float32),
                         s=s[None].astype(np.float32), payload=payload, M=M)
    d = np.array([0.3, -0.2, 1.0])
    d /= np.linalg.norm(d)
    o = np.array([0.05, 0.02, -3.0])
    dt = 0.01
    rays = rays_from(o, d, 0.0, 6.0, dt)
    out = orc.render(sc, rays, BRUTE64)["rgba"][0]
    o32, d32 = o.astype(np.float32).astype(np.float64), d.astype(np.float32).astype(np.float64)
    dt64 = float(np.float32(dt))
    A = 0.0
    I = np.zeros(3)
    for i in range(rays.n_steps):
        x = o32 + (i * dt64) * d32
        y = x / s.astype(np.float32)
        if np.max(np.abs(y)) > 1:
            continue
        u = (y + 1) / 2 * (M - 1)
        al = a0 + a @ u
        rgb = np.array([0.5, 0.1 * u[0], 0.1 * u[2]])
        A += dt64 * al
        I += dt64 * al * rgb
    assert A < 1
    assert abs(out[3] - A) < 1e-9
    np.testing.assert_allclose(out[:3], I, atol=1e-9)


# --------------------------------------------------------------------------- Sec. 3.2.1 hit lists
def test_ray_box_entry_exit_analytic(orc):
    """Entry/exit of rays through rotated, translated boxes equal those of the same
    configuration expressed in the box frame, where they are closed-form."""
    rng = np.random.default_rng(3)
    n = 50
    s = rng.uniform(0.2, 0.6, (n, 3))
    q = synthetic.random_unit_quaternions(rng, n)
    t = rng.uniform(-1, 1, (n, 3))
    # in the box frame: ray along local +x through (0, py, pz) with |py|,|pz| < 1 (scaled)
    py, pz = rng.uniform(-0.9, 0.9, n), rng.uniform(-0.9, 0.9, n)
    start = 3.0
    for k in range(n):
        R = rot_matrix(q[k])
        lo = np.array([-start, py[k] * s[k, 1], pz[k] * s[k, 2]])
        ld = np.array([1.0, 0.0, 0.0])
        o = t[k] + R @ lo
        d = R @ ld
        sc_t, sc_q, sc_s = t[k:k + 1], q[k:k + 1], s[k:k + 1]
        offs, ids, tin, tout, margin = orc.hit_lists(sc_t, sc_q, sc_s, o[None], d[None], 0.0, 10.0, "f64")
        assert offs[-1] == 1
        # closed form: enters at start - s_x, leaves at start + s_x
        assert abs(tin[0] - (start - s[k, 0])) < 2e-6
        assert abs(tout[0] - (start + s[k, 0])) < 2e-6
        offs, ids, tin32, tout32, _ = orc.hit_lists(sc_t, sc_q, sc_s, o[None], d[None], 0.0, 10.0, "f32")
        assert offs[-1] == 1
        assert abs(tin32[0] - tin[0]) < 2e-5 and abs(tout32[0] - tout[0]) < 2e-5


def test_ray_box_dense_sampling(orc):
    """Hit intervals agree with a dense inside test along each ray (brute force)."""
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 2)
    sel = np.arange(0, rays.n, 37)
    o, d = rays.o[sel], rays.d[sel]
    offs, ids, tin, tout, margin = orc.hit_lists(sc.t, sc.q, sc.s, o, d, 1.0, 5.0, "f64")
    R = rot_matrix(sc.q)
    ts = np.linspace(1.0, 5.0, 40001)
    h = ts[1] - ts[0]
    for r in range(len(sel)):
        x = o[r].astype(np.float64)[None] + ts[:, None] * d[r].astype(np.float64)[None]
        hits = {}
        for k in range(sc.n):
            y = ((x - sc.t[k]) @ R[k]) / sc.s[k]
            inside = np.max(np.abs(y), axis=1) <= 1
            if inside.any():
                hits[k] = (ts[inside][0], ts[inside][-1])
        got = {int(ids[j]): (tin[j], tout[j]) for j in range(offs[r], offs[r + 1]) if margin[j] >= 0}
        for k, (a, b) in hits.items():
            assert k in got
            assert got[k][0] <= a + 1e-12 and a - got[k][0] <= h + 1e-9
            assert got[k][1] >= b - 1e-12 and got[k][1] - b <= h + 1e-9
        for k, (a, b) in got.items():
            if k not in hits:
                assert b - a < h  # a chord shorter than the sampling step


def test_hit_sets_f32_equal_f64_except_grazing(orc):
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 0)
    o64 = orc.hit_lists(sc.t, sc.q, sc.s, rays.o, rays.d, rays.t_near, rays.t_far, "f64")
    o32 = orc.hit_lists(sc.t, sc.q, sc.s, rays.o, rays.d, rays.t_near, rays.t_far, "f32")
    offs64, ids64, _, _, m64 = o64
    offs32, ids32, tin32, tout32, _ = o32
    assert offs32[-1] > 5 * rays.n  # overlapping primitives: several hits per ray
    n_graze = 0
    for r in range(rays.n):
        s64 = {int(k): m for k, m in zip(ids64[offs64[r]:offs64[r + 1]], m64[offs64[r]:offs64[r + 1]])}
        hit64 = {k for k, m in s64.items() if m >= 0}
        graze = {k for k, m in s64.items() if abs(m) < 1e-4}
        hit32 = set(int(k) for k in ids32[offs32[r]:offs32[r + 1]])
        assert (hit32 ^ hit64) <= graze
        n_graze += len(graze)
    assert np.all(tin32 <= tout32)


# --------------------------------------------------------------------------- Sec. 3.2.2 invariants
@pytest.mark.parametrize("mode", ALL_MODES)
def test_empty_scene_returns_background(orc, mode):
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 0)
    rays.bg = (0.1, 0.2, 0.3)
    empty = synthetic.Scene(t=sc.t[:0], q=sc.q[:0], s=sc.s[:0], payload=sc.payload[:0], M=sc.M)
    out = orc.render(empty, rays, mode)["rgba"]
    np.testing.assert_array_equal(out[:, :3], np.broadcast_to(np.float32(rays.bg).astype(np.float64), (rays.n, 3)))
    assert np.all(out[:, 3] == 0)
    zero = synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, payload=np.zeros_like(sc.payload), M=sc.M)
    out = orc.render(zero, rays, mode)["rgba"]
    assert np.all(out[:, 3] == 0)


@pytest.mark.parametrize("mode", [PRUNED64, PRUNED32])
def test_permutation_invariance(orc, mode):
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 4)
    perm = np.random.default_rng(0).permutation(sc.n)
    a = orc.render(sc, rays, mode)["rgba"]
    b = orc.render(permute_scene(sc, perm), rays, mode)["rgba"]
    np.testing.assert_allclose(a, b, atol=1e-12)
    h1 = orc.hit_lists(sc.t, sc.q, sc.s, rays.o, rays.d, 1.0, 5.0, "f32")
    ps = permute_scene(sc, perm)
    h2 = orc.hit_lists(ps.t, ps.q, ps.s, rays.o, rays.d, 1.0, 5.0, "f32")
    np.testing.assert_array_equal(h1[0], h2[0])
    for r in range(0, rays.n, 97):
        s1 = set(h1[1][h1[0][r]:h1[0][r + 1]].tolist())
        s2 = set(perm[h2[1][h2[0][r]:h2[0][r + 1]]].tolist())
        assert s1 == s2


def test_rigid_invariance(orc):
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 5)
    G = rot_matrix([0.8, 0.1, -0.5, 0.3])
    b = np.array([0.4, -1.1, 2.0])
    R = rot_matrix(sc.q)
    sc2 = synthetic.Scene(t=(sc.t.astype(np.float64) @ G.T + b).astype(np.float32),
                          q=quat_from_matrix(G[None] @ R).astype(np.float32), s=sc.s, payload=sc.payload,
                          M=sc.M)
    r2 = rays_from((rays.o.astype(np.float64) @ G.T + b), rays.d.astype(np.float64) @ G.T,
                   rays.t_near, rays.t_far, rays.dt)
    a = orc.render(sc, rays, PRUNED64)
    c = orc.render(sc2, r2, PRUNED64)
    ok = ~(a["near_face"] | c["near_face"])
    assert ok.mean() > 0.95
    np.testing.assert_allclose(a["rgba"][ok], c["rgba"][ok], atol=2e-5)


def test_saturation_hides_content_behind(orc):
    """Once T reaches 1 nothing behind contributes (Sec. 3.2.2, early stop)."""
    front = single_box(M=3, alpha=50.0, rgb=(0.9, 0.1, 0.2), t=(0, 0, 0), s=(0.3, 0.3, 0.3))
    back_a = single_box(M=3, alpha=2.0, rgb=(0.1, 0.8, 0.3), t=(0, 0, 1.0), s=(0.3, 0.3, 0.3))
    back_b = single_box(M=3, alpha=7.0, rgb=(0.5, 0.5, 0.5), t=(0.05, 0, 1.2), s=(0.35, 0.3, 0.3))
    rays = rays_from([0, 0, -3], [[0, 0, 1], [0.02, 0.01, 1]], 0.0, 8.0, 0.005)
    rays.d = (rays.d / np.linalg.norm(rays.d, axis=1, keepdims=True)).astype(np.float32)
    a = orc.render(concat_scenes(front, back_a), rays, PRUNED64)
    b = orc.render(concat_scenes(front, back_b), rays, PRUNED64)
    assert np.all(a["rgba"][:, 3] == 1.0)
    np.testing.assert_array_equal(a["rgba"], b["rgba"])
    np.testing.assert_allclose(a["rgba"][:, :3], np.broadcast_to([0.9, 0.1, 0.2], (2, 3)), atol=1e-6)


def test_early_stop_error_bound(orc):
    """Stopping at T >= 1 - eps changes every channel by at most eps (the remaining
    weights sum to at most eps and colours lie in [0, 1])."""
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 1)
    ref = orc.render(sc, rays, PRUNED32)["rgba"]
    for eps in (0.01, 0.1):
        rays.eps_early = eps
        out = orc.render(sc, rays, PRUNED32)["rgba"]
        assert np.max(np.abs(out - ref)) <= eps + 1e-9
        assert np.all(out[:, 3] <= ref[:, 3] + 1e-12)
    rays.eps_early = 0.0


def test_background_composite(orc):
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 3)
    a = orc.render(sc, rays, PRUNED32)["rgba"]
    rays.bg = (0.25, 0.5, 1.0)
    b = orc.render(sc, rays, PRUNED32)["rgba"]
    bg = np.float32(rays.bg).astype(np.float64)
    np.testing.assert_allclose(b[:, :3], a[:, :3] + (1 - a[:, 3:4]) * bg[None], atol=1e-12)
    np.testing.assert_array_equal(a[:, 3], b[:, 3])


def test_order_free_sum_within_sample(orc):
    """Two coincident primitives give the image of one primitive with the summed
    payload wherever no clamp happens (R2: summed, then clamped once)."""
    rng = np.random.default_rng(9)
    M = 4
    p1 = rng.random((1, M, M, M, 4)).astype(np.float32) * 0.5
    p2 = rng.random((1, M, M, M, 4)).astype(np.float32) * 0.5
    base = dict(t=np.zeros((1, 3), np.float32), q=np.array([[1, 0, 0, 0]], np.float32),
                s=np.full((1, 3), 0.4, np.float32), M=M)
    two = synthetic.Scene(t=np.repeat(base["t"], 2, 0), q=np.repeat(base["q"], 2, 0),
                          s=np.repeat(base["s"], 2, 0), payload=np.concatenate([p1, p2]), M=M)
    summed = p1 + p2
    summed[..., :3] = (p1[..., 3:] * p1[..., :3] + p2[..., 3:] * p2[..., :3]) / np.maximum(summed[..., 3:], 1e-30)
    # colour is alpha-weighted, so only equal for constant colour fields: use a constant-colour case
    p1[..., :3] = 0.3
    p2[..., :3] = 0.3
    two.payload = np.concatenate([p1, p2])
    one = synthetic.Scene(payload=(np.concatenate([p1[..., :3], p1[..., 3:] + p2[..., 3:]], -1)), **base)
    d = rng.standard_normal((64, 3))
    d[:, 2] = np.abs(d[:, 2]) + 6
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = rays_from([0, 0, -3], d, 0.0, 6.0, 0.01)
    a = orc.render(two, rays, BRUTE64)["rgba"]
    b = orc.render(one, rays, BRUTE64)["rgba"]
    assert np.all(a[:, 3] < 1)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_literal_composite(orc):
    """Mode bit 3 reads the composite as A I + (1 - A) B (Sec. 3.1.4 printed literally):
    on the uniform box I = c A, so the literal reading gives c A^2 + (1 - A) B; on a
    scene, only the background composite changes."""
    g = json.load(open(os.path.join(GOLDEN, "uniform_box.json")))
    b, r = g["box"], g["ray"]
    bg = (0.25, 0.5, 1.0)
    for case in g["cases"]:
        sc = single_box(M=b["M"], alpha=case["sigma"], rgb=b["rgb"], t=b["t"], q=b["q"], s=b["s"])
        rays = rays_from(r["o"], r["d"], r["t_near"], r["t_far"], r["dt"], eps=case["eps"], bg=bg)
        out = orc.render(sc, rays, PRUNED64 | 8)["rgba"][0]
        A = case["A"]
        expect = np.float32(b["rgb"]).astype(np.float64) * A * A + (1 - A) * np.float32(bg).astype(np.float64)
        assert abs(out[3] - A) < g["tolerance"]
        np.testing.assert_allclose(out[:3], expect, atol=2 * g["tolerance"])
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 3)
    rays.bg = bg
    pre = orc.render(sc, rays, PRUNED32)["rgba"]
    lit = orc.render(sc, rays, PRUNED32 | 8)["rgba"]
    B = np.float32(bg).astype(np.float64)[None]
    A = pre[:, 3:4]
    np.testing.assert_array_equal(lit[:, 3], pre[:, 3])
    np.testing.assert_allclose(lit[:, :3], A * (pre[:, :3] - (1 - A) * B) + (1 - A) * B, atol=1e-12)
    assert np.abs(lit - pre).max() > 1e-3


# --------------------------------------------------------------------------- modes agree
@pytest.mark.parametrize("member", [0, 2])
def test_brute_equals_pruned(orc, member):
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 0)
    a = orc.render(sc, rays, 0 | member)
    b = orc.render(sc, rays, 1 | member)
    np.testing.assert_array_equal(a["rgba"], b["rgba"])
    np.testing.assert_array_equal(a["n_eval"], b["n_eval"])
    np.testing.assert_array_equal(a["near_face"], b["near_face"])


def test_f32_membership_differs_only_near_faces(orc):
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 1)
    a = orc.render(sc, rays, PRUNED64)
    b = orc.render(sc, rays, PRUNED32)
    diff = np.abs(a["rgba"] - b["rgba"]).max(1)
    # away from faces only the float32 sample time differs (~1e-7 relative)
    assert np.all(diff[~a["near_face"]] < 2e-5)


# --------------------------------------------------------------------------- LBVH keys and tree
def _deinterleave(m):
    b = format(int(m), "030b")
    return int(b[0::3], 2), int(b[1::3], 2), int(b[2::3], 2)


def test_morton_keys(orc):
    rng = np.random.default_rng(11)
    t = rng.normal(0, 1, (500, 3)).astype(np.float32)
    t[7] = t[3]  # duplicate centre
    bounds, keys = orc.morton_keys(t)
    np.testing.assert_array_equal(bounds[:3], t.min(0))
    np.testing.assert_array_equal(bounds[3:], t.max(0))
    assert np.all((keys & np.uint64(0xFFFFFFFF)) == np.arange(500, dtype=np.uint64))
    codes = (keys >> np.uint64(32)).astype(np.int64)
    qs = np.array([_deinterleave(c) for c in codes])
    assert qs.min() == 0 and qs.max() == 1023
    for j in range(3):
        assert qs[np.argmin(t[:, j]), j] == 0 and qs[np.argmax(t[:, j]), j] == 1023
        # quantisation is monotone in the coordinate and within one cell of the exact value
        order = np.argsort(t[:, j], kind="stable")
        assert np.all(np.diff(qs[order, j]) >= 0)
        u = (t[:, j].astype(np.float64) - bounds[j]) / (float(bounds[3 + j]) - float(bounds[j]))
        assert np.all(np.abs(qs[:, j] - np.minimum(np.floor(u * 1024), 1023)) <= 1)
    assert codes[7] == codes[3]
    # all centres equal: every code is 0, keys still unique
    _, k0 = orc.morton_keys(np.ones((5, 3), np.float32))
    assert np.all((k0 >> np.uint64(32)) == 0) and len(set(k0.tolist())) == 5


def _radix_tree_bruteforce(keys):
    """Independent construction on binary strings: split each range at the first key
    whose string differs from the range's first key at the range's common-prefix length."""
    s = [format(int(k), "064b") for k in keys]
    n = len(s)
    left, right = [None] * (n - 1), [None] * (n - 1)

    def rec(a, b, node):
        pre = len(os.path.commonprefix([s[a], s[b]]))
        g = max(i for i in range(a, b) if s[i][pre] == "0")
        left[node] = g if g > a else n - 1 + g
        right[node] = g + 1 if g + 1 < b else n - 1 + g + 1
        if g > a:
            rec(a, g, g)
        if g + 1 < b:
            rec(g + 1, b, g + 1)

    if n >= 2:
        rec(0, n - 1, 0)
    return np.array(left, np.int64), np.array(right, np.int64)


@pytest.mark.parametrize("n", [2, 3, 17, 300])
def test_radix_tree_matches_bruteforce(orc, n):
    rng = np.random.default_rng(n)
    t = rng.normal(0, 1, (n, 3)).astype(np.float32)
    if n > 10:
        t[5:9] = t[2]  # equal Morton codes are separated by the index bits
    _, keys = orc.morton_keys(t)
    sk = np.sort(keys)
    left, right = orc.radix_tree(sk)
    bl, br = _radix_tree_bruteforce(sk)
    np.testing.assert_array_equal(left, bl)
    np.testing.assert_array_equal(right, br)
    # every node except the root has exactly one parent
    children = np.concatenate([left, right])
    assert sorted(children.tolist()) == list(range(1, 2 * n - 1))


# --------------------------------------------------------------------------- inputs
def test_inputs_deterministic_and_shaped():
    a = synthetic.make_config("tiny_8x8^3_64x64", 3)
    b = synthetic.make_config("tiny_8x8^3_64x64", 3)
    np.testing.assert_array_equal(a[0].payload, b[0].payload)
    np.testing.assert_array_equal(a[1].d, b[1].d)
    sc, rays, _ = a
    assert sc.payload.shape == (8, 8, 8, 8, 4) and rays.o.shape == (4096, 3)
    assert rays.n_steps == 400
    np.testing.assert_allclose(np.linalg.norm(rays.d, axis=1), 1.0, atol=1e-6)
    assert abs((sc.payload[..., 3] == 0).mean() - 0.5) < 0.03
    assert np.allclose(np.linalg.norm(sc.t, axis=1), 1.0, atol=1e-6)


def test_paper_scale_inputs_follow_the_recipe():
    """The benchmark frame's inputs: 4096 primitives of 16^3 on an ellipsoid shell of radii
    (1, 1.2, 0.9) with N(0, 0.02^2) jitter, half extents U[0.04, 0.08], 60 % empty voxels,
    alpha = 4 softplus(N(0, 1)), one 667x1024 camera at radius 3 looking at the centre,
    dt = 0.005 over [1, 5] (800 samples); the differentiation workload adds the opacity
    fade window and four 512x512 cameras with a seeded target."""
    sc, rays, _ = synthetic.make_config("paper_4096x16^3_667x1024", 0)
    assert sc.payload.shape == (4096, 16, 16, 16, 4) and sc.payload.dtype == np.float32
    assert rays.o.shape == (683008, 3) and (rays.width, rays.height) == (667, 1024)
    assert rays.n_steps == 800 and (rays.t_near, rays.t_far, rays.dt) == (1.0, 5.0, 0.005)
    assert sc.s.min() >= 0.04 and sc.s.max() <= 0.08
    np.testing.assert_allclose(np.linalg.norm(sc.q, axis=1), 1.0, atol=1e-6)
    radial = np.linalg.norm(sc.t / np.float32([1.0, 1.2, 0.9]), axis=1)
    assert abs(np.median(radial) - 1.0) < 0.01 and radial.min() > 0.85 and radial.max() < 1.15
    a = sc.payload[..., 3]
    empty = (sc.payload == 0).all(-1)
    assert abs(empty.mean() - 0.6) < 0.005
    # mean of 4 softplus(z) over the occupied voxels: 4 E[softplus(N(0,1))] = 3.226
    assert abs(a[~empty].mean() - 3.226) < 0.01
    np.testing.assert_allclose(np.linalg.norm(rays.o[0]), 3.0, rtol=1e-6)
    centre = rays.d[(1024 // 2) * 667 + 667 // 2]
    np.testing.assert_allclose(centre, -rays.o[0] / 3.0, atol=2e-3)
    sc3, rays3, extra = synthetic.make_config("diff_512x32^3_4x512x512", 0)
    assert sc3.payload.shape == (512, 32, 32, 32, 4) and rays3.n == 4 * 512 * 512
    assert extra["target"].shape == (rays3.n, 3)
    # the fade window leaves the centre voxel's opacity (nearly) whole and zeroes the corners
    occupied = sc3.payload[..., 3] > 0
    assert sc3.payload[:, 0, 0, 0, 3].max() < 1e-6 * sc3.payload[..., 3].max()
    assert occupied[:, 15:17, 15:17, 15:17].mean() > 0.3
