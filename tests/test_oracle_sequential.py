"""Pins of the oracle's sequential blending mode (primitives that share a sample taken
one by one in BVH order, Sec. 3.2.2) against closed forms and invariances.

The BVH order is the leaf order of the Karras hierarchy: ascending Morton keys of the
primitive centres. The two blending rules agree wherever T stays below 1, so they may
differ only at a ray's saturating sample.
"""
import numpy as np
import pytest

import synthetic
from helpers import concat_scenes, permute_scene, rays_from, single_box

SEQ = 4
PRUNED32 = 3
MODES = [0, 1, 2, 3]


def _pair(x_first, x_second, a1, a2, c1, c2):
    """Two boxes that both contain the ray x = y = 0 over z in [-0.3, 0.3]; box i sits
    at x = x_i. The scene lists them in the given order."""
    p = single_box(M=3, alpha=a1, rgb=c1, t=(x_first, 0, 0), s=(0.3, 0.3, 0.3))
    q = single_box(M=3, alpha=a2, rgb=c2, t=(x_second, 0, 0), s=(0.3, 0.3, 0.3))
    return concat_scenes(p, q)


@pytest.mark.parametrize("mode", MODES)
def test_saturating_sample_in_morton_order_closed_form(orc, mode):
    """Constant fields, alpha dt = 0.17 and 0.19: two full samples give T = 0.72, the
    third saturates with 1 - T = 0.28. The primitive at lower x has the lower Morton
    key (the centres differ only in x), so it blends first, whatever its index."""
    dt = 0.01
    aA, aB = 17.0, 19.0
    cA, cB = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.7, 0.4])
    # first sample inside: t = 0.0037 + 0.01 i >= 2.7 at i = 270 (no sample near a face)
    rays = rays_from([0, 0, -3], [0, 0, 1], 0.0037, 6.0, dt)
    cA32, cB32 = cA.astype(np.float32).astype(np.float64), cB.astype(np.float32).astype(np.float64)
    full = 2 * dt * (aA * cA32 + aB * cB32)
    rem = 1.0 - 2 * dt * (aA + aB)
    for xa, xb, listed_a_first in ((-0.05, 0.05, True), (0.05, -0.05, True), (-0.05, 0.05, False)):
        if listed_a_first:
            sc = _pair(xa, xb, aA, aB, cA, cB)
        else:
            sc = _pair(xb, xa, aB, aA, cB, cA)
        out = orc.render(sc, rays, mode | SEQ)
        first, second = ((aA, cA32), (aB, cB32)) if xa < xb else ((aB, cB32), (aA, cA32))
        w1 = min(dt * first[0], rem)
        w2 = min(dt * second[0], rem - w1)
        expect = full + first[1] * w1 + second[1] * w2
        np.testing.assert_allclose(out["rgba"][0, :3], expect, atol=1e-12)
        assert out["rgba"][0, 3] == 1.0
        assert out["i_clamp"][0] == 272
        # the summed rule on the same scene: c * (1 - T) / a at the clamp
        summ = orc.render(sc, rays, mode)
        expect_sum = full + (rem / (dt * (aA + aB))) * dt * (aA * cA32 + aB * cB32)
        np.testing.assert_allclose(summ["rgba"][0, :3], expect_sum, atol=1e-12)
        assert np.abs(summ["rgba"][0, :3] - out["rgba"][0, :3]).max() > 1e-3


def test_rules_agree_off_the_saturating_sample(orc):
    """Rays that never saturate, and the opacity of every ray, are identical; the
    difference on a saturating ray is bounded by (1 - T) at its clamp, colours in [0, 1]."""
    for seed in range(3):
        sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", seed)
        a = orc.render(sc, rays, PRUNED32)
        b = orc.render(sc, rays, PRUNED32 | SEQ)
        np.testing.assert_array_equal(a["i_clamp"], b["i_clamp"])
        free = a["i_clamp"] < 0
        np.testing.assert_array_equal(a["rgba"][free], b["rgba"][free])
        np.testing.assert_array_equal(a["rgba"][:, 3], b["rgba"][:, 3])
        assert np.all(np.abs(a["rgba"] - b["rgba"]) <= 1.0 + 1e-12)
        assert np.any(np.abs(a["rgba"] - b["rgba"]) > 1e-6)  # the scene has saturating overlaps


def test_single_primitive_saturation_equals_summed(orc):
    """With one primitive at the saturating sample both rules add c (1 - T)."""
    sc = single_box(M=3, alpha=30.0, rgb=(0.3, 0.6, 0.9), s=(0.3, 0.3, 0.3))
    d = np.random.default_rng(2).standard_normal((32, 3)) * 0.02 + [0, 0, 1]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = rays_from([0, 0, -3], d, 0.0, 6.0, 0.0123)
    a = orc.render(sc, rays, PRUNED32)["rgba"]
    b = orc.render(sc, rays, PRUNED32 | SEQ)["rgba"]
    assert np.all(a[:, 3] == 1.0)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_sequential_order_follows_positions_not_indices(orc):
    """Relabelling the primitives leaves the BVH order, hence the image, unchanged."""
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 4)
    perm = np.random.default_rng(0).permutation(sc.n)
    a = orc.render(sc, rays, PRUNED32 | SEQ)["rgba"]
    b = orc.render(permute_scene(sc, perm), rays, PRUNED32 | SEQ)["rgba"]
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_sequential_brute_equals_pruned(orc):
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 0)
    a = orc.render(sc, rays, 2 | SEQ)["rgba"]
    b = orc.render(sc, rays, 3 | SEQ)["rgba"]
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_sequential_adjoint_closed_form(orc):
    """The two-box scene, loss g . I: box A (lower x, first in BVH order) enters the
    saturating sample whole, box B is clamped to what is left. Summed over each box's
    voxels (a constant field: the trilinear weights of a sample sum to 1):
    dL/dalpha_A = 3 dt g.(c_A - c_B), dL/dalpha_B = 0, dL/dc_A = 3 dt alpha_A g,
    dL/dc_B = (2 dt alpha_B + w_B) g with w_B = 1 - 2 dt (alpha_A + alpha_B) - dt alpha_A."""
    dt, aA, aB = 0.01, 17.0, 19.0
    cA, cB = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.7, 0.4])
    rays = rays_from([0, 0, -3], [0, 0, 1], 0.0037, 6.0, dt)
    sc = _pair(0.05, -0.05, aB, aA, cB, cA)  # listed B first: the order must come from the positions
    g = np.array([[0.3, -1.2, 0.7, 0.4]])
    G = orc.backward(sc, rays, g, 3 | SEQ)["g_payload"]
    cA32, cB32 = cA.astype(np.float32).astype(np.float64), cB.astype(np.float32).astype(np.float64)
    wB = 1 - 2 * dt * (aA + aB) - dt * aA
    gB, gA = G[0].reshape(-1, 4).sum(0), G[1].reshape(-1, 4).sum(0)  # scene order: B, A
    np.testing.assert_allclose(gA[3], 3 * dt * g[0, :3] @ (cA32 - cB32), atol=1e-12)
    assert abs(gB[3]) < 1e-12
    np.testing.assert_allclose(gA[:3], 3 * dt * aA * g[0, :3], atol=1e-12)
    np.testing.assert_allclose(gB[:3], (2 * dt * aB + wB) * g[0, :3], atol=1e-12)
    # the summed rule on the same scene gives other values (it treats both boxes alike)
    Gs = orc.backward(sc, rays, g, 3)["g_payload"]
    assert abs(Gs[0].reshape(-1, 4).sum(0)[3]) > 1e-3


def test_sequential_adjoint_matches_finite_differences(orc):
    """Payload gradients of the sequential mode against central differences of its own
    forward (the image is piecewise linear in the payload), on a scene where the rule
    matters."""
    from helpers import zero_boundary

    sc, rays, _ = synthetic.make_config("diff_small_64x8^3_2x48x40", 1)
    sc = zero_boundary(sc)
    g = np.random.default_rng(6).standard_normal((rays.n, 4))
    diff = np.abs(orc.render(sc, rays, 3 | SEQ)["rgba"] - orc.render(sc, rays, 3)["rgba"]).max()
    assert diff > 1e-4  # the scene has saturating samples shared by several primitives
    gp = orc.backward(sc, rays, g, 3 | SEQ)["g_payload"]
    scale = np.abs(gp).max()

    def loss(P):
        return float((orc.render(synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, payload=P, M=sc.M), rays,
                                 3 | SEQ)["rgba"] * g).sum())

    rng = np.random.default_rng(2)
    nz = np.argwhere(np.abs(gp) > 1e-3 * scale)
    for j in rng.choice(len(nz), 16, replace=False):
        idx = tuple(nz[j])
        a, b = sc.payload.copy(), sc.payload.copy()
        a[idx] += 1e-3
        b[idx] -= 1e-3
        f = (loss(a) - loss(b)) / (float(a[idx]) - float(b[idx]))
        assert abs(f - gp[idx]) <= 1e-6 * scale, (idx, f, gp[idx])


def test_sequential_composes_with_the_literal_background(orc):
    """The two ray flags act on different steps: the sequential rule changes the
    saturating sample's blend, the literal reading only the background composite
    (Sec. 3.1.4). Together, the image is the literal composite of the sequential result."""
    sc, rays, _ = synthetic.make_config("tiny_8x8^3_64x64", 2)
    bg = (0.25, 0.5, 1.0)
    rays.bg = bg
    seq = orc.render(sc, rays, PRUNED32 | SEQ)["rgba"]
    both = orc.render(sc, rays, PRUNED32 | SEQ | 8)["rgba"]
    B = np.float32(bg).astype(np.float64)[None]
    A = seq[:, 3:4]
    np.testing.assert_array_equal(both[:, 3], seq[:, 3])
    np.testing.assert_allclose(both[:, :3], A * (seq[:, :3] - (1 - A) * B) + (1 - A) * B, atol=1e-12)
    summed_literal = orc.render(sc, rays, PRUNED32 | 8)["rgba"]
    assert np.abs(both - summed_literal).max() > 1e-4
