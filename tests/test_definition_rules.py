"""CPU checks of the parity rules against the FP64 definition (tests/parity_rules.py).

The oracle's FP32 decision mode (the operation order the CUDA path follows for its
membership and hit decisions) must meet the same bar against the oracle's FP64
definition that the GPU tests apply, and planted mistakes must fail it.
"""
import numpy as np
import pytest

import oracle
import synthetic
from helpers import rays_from
from parity_rules import definition_bar, hit_sets_vs_f64

F32M = oracle.MODE_PRUNED | oracle.MEMBER_F32
F64M = oracle.MODE_PRUNED | oracle.MEMBER_F64


@pytest.mark.parametrize("cfg", ["tiny_8x8^3_64x64", "small_512x8^3_96x128", "small_4096x16^3_83x128"])
def test_fp32_spec_meets_the_definition_bar(cfg):
    sc, rays, _ = synthetic.make_config(cfg, 0)
    f32 = oracle.render(sc, rays, F32M)
    f64 = oracle.render(sc, rays, F64M)
    definition_bar(f32["rgba"], f64, cfg)
    hit_sets_vs_f64(oracle.hit_lists(sc.t, sc.q, sc.s, rays.o, rays.d, rays.t_near, rays.t_far, "f32")[:4],
                    oracle.hit_lists(sc.t, sc.q, sc.s, rays.o, rays.d, rays.t_near, rays.t_far, "f64"), sc, rays, cfg)


def test_definition_bar_rejects_planted_errors():
    sc, rays, _ = synthetic.make_config("small_512x8^3_96x128", 0)
    f64 = oracle.render(sc, rays, F64M)
    img = f64["rgba"].copy()
    far = np.flatnonzero(~f64["near_face"])
    bad = img.copy()
    bad[far[7], 1] += 3e-4  # one channel off the band on a pixel no face explains
    with pytest.raises(AssertionError):
        definition_bar(bad, f64, "planted off-face error")
    bad = img.copy()
    near = np.flatnonzero(f64["near_face"])
    bad[near[3], 2] += 0.15  # near a face, but above the near-face cap
    with pytest.raises(AssertionError):
        definition_bar(bad, f64, "planted error above the cap")
    bad = img.copy()
    bad[near[3:20], 2] += 2e-2  # near faces, but over 1e-2 on more than 1 % of the near-face pixels
    with pytest.raises(AssertionError):
        definition_bar(bad, f64, "planted errors over 1e-2")
    bad = img.copy()
    bad[near[:60], :3] += 5e-4  # near faces, but more than 0.1 % of channels off the band
    with pytest.raises(AssertionError):
        definition_bar(bad, f64, "planted widespread error")
    ok = img.copy()
    ok[near[5], 0] += 5e-3  # near a face, under the cap: allowed
    definition_bar(ok, f64, "allowed near-face error")


def test_hit_set_rule_rejects_planted_errors():
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 0)
    f64 = oracle.hit_lists(sc.t, sc.q, sc.s, rays.o, rays.d, rays.t_near, rays.t_far, "f64")
    offs, ids, tin, tout, margin = f64
    hit = margin >= 0
    # the FP64 hits themselves pass
    ray = np.repeat(np.arange(rays.n), np.diff(offs))
    cnt = np.bincount(ray[hit], minlength=rays.n)
    g_offs = np.concatenate([[0], np.cumsum(cnt)])
    gl = (g_offs, ids[hit], tin[hit].astype(np.float32), tout[hit].astype(np.float32))
    hit_sets_vs_f64(gl, f64, sc, rays, "FP64 hits")
    # dropping a pair that is not grazing fails
    keep = np.ones(int(hit.sum()), bool)
    wide = np.flatnonzero(margin[hit] > 1e-2)
    keep[wide[0]] = False
    r = np.searchsorted(g_offs, wide[0], side="right") - 1
    cnt2 = cnt.copy()
    cnt2[r] -= 1
    g2 = (np.concatenate([[0], np.cumsum(cnt2)]), gl[1][keep], gl[2][keep], gl[3][keep])
    with pytest.raises(AssertionError):
        hit_sets_vs_f64(g2, f64, sc, rays, "dropped pair")
    # a shifted interval fails
    g3 = (gl[0], gl[1], gl[2] + np.float32(3e-4), gl[3])
    with pytest.raises(AssertionError):
        hit_sets_vs_f64(g3, f64, sc, rays, "shifted interval")


def test_grazing_rays_differ_only_by_grazing_pairs():
    """Rays aimed at box corners and edge midpoints: the FP32 spec's hit sets differ from
    the FP64 ones, if at all, only by pairs the rule calls grazing."""
    rng = np.random.default_rng(5)
    sc = synthetic.make_scene(300, 4, 3, layout="shell", s_range=(0.05, 0.2))
    n = 1000
    o = rng.normal(0, 3, (n, 3))
    target = np.zeros((n, 3))
    R = oracle.rotations(sc.q)
    for i in range(n):
        k = rng.integers(0, sc.n)
        y = rng.choice([-1.0, 1.0], 3)
        if i % 2 == 0:
            y[rng.integers(0, 3)] = 0.0
        target[i] = sc.t[k] + R[k] @ (y * sc.s[k])
    d = target - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = rays_from(o, d, 0.5, 9.0, 0.01)
    st = hit_sets_vs_f64(oracle.hit_lists(sc.t, sc.q, sc.s, rays.o, rays.d, 0.5, 9.0, "f32")[:4],
                         oracle.hit_lists(sc.t, sc.q, sc.s, rays.o, rays.d, 0.5, 9.0, "f64"), sc, rays, "corners")
    assert st["pairs_f64"] > n // 2


@pytest.mark.parametrize("cfg", ["paper_4096x16^3_667x1024", "sweep_512x32^3_667x1024"])
def test_fp32_spec_meets_the_definition_bar_at_paper_scale(cfg):
    sc, rays, _ = synthetic.make_config(cfg, 0)
    sel = np.random.default_rng(7).choice(rays.n, 3000, replace=False)
    sub = rays_from(rays.o[sel], rays.d[sel], rays.t_near, rays.t_far, rays.dt)
    definition_bar(oracle.render(sc, sub, F32M)["rgba"], oracle.render(sc, sub, F64M), cfg)


def test_fp32_spec_adjoint_differs_from_the_definition_only_on_face_voxels():
    """The two membership decisions give the same gradients except the opacity gradients
    of voxels on a box face (where a sample on the face is in by one decision and out by
    the other)."""
    sc, rays, _ = synthetic.make_config("diff_small_64x8^3_2x48x40", 0)
    g = np.random.default_rng(3).standard_normal((rays.n, 4))
    a = oracle.backward(sc, rays, g, F32M)
    b = oracle.backward(sc, rays, g, F64M)
    M = sc.M
    face = np.zeros((M, M, M), bool)
    face[[0, -1]] = True
    face[:, [0, -1]] = True
    face[:, :, [0, -1]] = True
    scale = np.abs(b["g_payload"]).max()
    assert np.abs(a["g_payload"][:, ~face] - b["g_payload"][:, ~face]).max() <= 1e-5 * scale
    assert np.abs(a["g_payload"][:, face, :3] - b["g_payload"][:, face, :3]).max() <= 1e-5 * scale
    assert np.abs(a["g_payload"][:, face, 3] - b["g_payload"][:, face, 3]).max() <= 1e-2 * scale
    for key in ("g_t", "g_q", "g_s"):
        assert np.abs(a[key] - b[key]).max() <= 1e-4 * np.abs(b[key]).max()
