"""Pins of the oracle's adjoint against central finite differences of its own FP64
forward (two independent computations: the forward never uses the adjoint's
formulas). The loss is L = sum(g * out) for a seeded g, so dL/dout = g.

Payload gradients are exact (the image is piecewise linear in the payload). Pose
gradients are piecewise smooth: the field has kinks at voxel-cell boundaries and at
box faces. A finite difference that straddles a kink is wrong by O(h) and is told apart
by comparing two step sizes; such parameters are counted and reported, and only
parameters whose two estimates agree are held to the tight tolerance.
"""
import numpy as np
import pytest

import synthetic
from helpers import rays_from, zero_boundary

MODE = 3  # pruned, FP32 membership (the mode the CUDA path is compared against)


def _setup(eps=0.0, bg=(0, 0, 0), seed=0):
    sc, rays, _ = synthetic.make_config("diff_small_64x8^3_2x48x40", seed)
    sc = zero_boundary(sc)
    rays.eps_early = eps
    rays.bg = bg
    g = np.random.default_rng(seed + 5).standard_normal((rays.n, 4))
    return sc, rays, g


def _loss(orc, sc, rays, g):
    return float((orc.render(sc, rays, MODE)["rgba"] * g).sum())


def _fd(orc, sc, rays, g, field, idx, h):
    a = getattr(sc, field).copy()
    b = a.copy()
    a[idx] += h
    b[idx] -= h
    sa = synthetic.Scene(**{**sc.__dict__, field: a})
    sb = synthetic.Scene(**{**sc.__dict__, field: b})
    return (_loss(orc, sa, rays, g) - _loss(orc, sb, rays, g)) / (float(a[idx]) - float(b[idx]))


@pytest.mark.parametrize("eps,bg", [(0.0, (0, 0, 0)), (0.05, (0.2, 0.5, 0.9))])
def test_payload_gradient_exact(orc, eps, bg):
    sc, rays, g = _setup(eps, bg)
    G = orc.backward(sc, rays, g, MODE)
    out = orc.render(sc, rays, MODE)
    if eps == 0.0:
        assert (out["i_clamp"] >= 0).sum() > 20  # the saturating-sample branch is exercised
    gp = G["g_payload"]
    scale = np.abs(gp).max()
    rng = np.random.default_rng(1)
    nz = np.argwhere(np.abs(gp) > 1e-3 * scale)
    picks = [tuple(nz[j]) for j in rng.choice(len(nz), 12, replace=False)]
    picks += [tuple(np.argwhere(gp == 0)[0])]
    for idx in picks:
        f = _fd(orc, sc, rays, g, "payload", idx, 1e-3)
        assert abs(f - gp[idx]) <= 1e-6 * scale, (idx, f, gp[idx])


def test_pose_gradient_single_sample_exact(orc):
    """One sample per ray, placed inside a box away from faces and voxel-cell
    boundaries: a small step crosses no kink, so central differences are exact to
    O(h^2) and pin the chain rule through y = diag(1/s) R(q)^T (x - t)."""
    rng = np.random.default_rng(4)
    M, n = 4, 3
    t = np.array([[-1.5, 0, 0], [0, 0.2, 0], [1.5, -0.1, 0.3]], np.float32)
    q = synthetic.random_unit_quaternions(rng, n)
    s = rng.uniform(0.3, 0.6, (n, 3)).astype(np.float32)
    payload = rng.random((n, M, M, M, 4)).astype(np.float32)
    sc = synthetic.Scene(t=t, q=q, s=s, payload=payload, M=M)
    Rm = orc.rotations(q)
    os_, ds_ = [], []
    for k in range(n):
        for _ in range(20):
            while True:
                u = rng.uniform(0.1, M - 1.1, 3)
                if np.all(np.abs(u - np.round(u)) > 0.08):
                    break
            y = u / (M - 1) * 2 - 1
            x = t[k].astype(np.float64) + Rm[k] @ (y * s[k])
            d = rng.standard_normal(3)
            d /= np.linalg.norm(d)
            os_.append(x - 2.0 * d)
            ds_.append(d)
    rays = rays_from(np.array(os_), np.array(ds_), 2.0, 2.0005, 1e-3)
    assert rays.n_steps == 1
    g = rng.standard_normal((rays.n, 4))
    G = orc.backward(sc, rays, g, 1)
    for field, key in (("t", "g_t"), ("q", "g_q"), ("s", "g_s")):
        gg = G[key]
        scale = np.abs(gg).max()
        assert scale > 0
        for k in range(n):
            for c in range(gg.shape[1]):
                f = _fd(orc, sc, rays, g, field, (k, c), 1e-4)
                assert abs(f - gg[k, c]) <= 1e-6 * scale, (field, k, c, f, gg[k, c])


def test_pose_gradient_scene_fd(orc):
    """Whole-scene finite differences: most parameters see no kink inside a 1e-6 step
    and match tightly; the rest are off by at most a few kink contributions."""
    sc, rays, g = _setup()
    G = orc.backward(sc, rays, g, MODE)
    rel = []
    for field, key in (("t", "g_t"), ("q", "g_q"), ("s", "g_s")):
        gg = G[key]
        scale = np.abs(gg).max()
        for k in range(0, sc.n, 13):
            for c in range(gg.shape[1]):
                f = _fd(orc, sc, rays, g, field, (k, c), 1e-6)
                rel.append(abs(f - gg[k, c]) / scale)
    rel = np.array(rel)
    assert np.median(rel) < 1e-6, np.sort(rel)
    assert rel.max() < 2e-2, np.sort(rel)


def test_quaternion_gradient_orthogonal_to_q(orc):
    """L depends on q only through q/|q|, so dL/dq is orthogonal to q."""
    sc, rays, g = _setup(seed=1)
    G = orc.backward(sc, rays, g, MODE)
    q = sc.q.astype(np.float64)
    dots = np.abs((G["g_q"] * q).sum(1))
    assert np.all(dots <= 1e-9 * (np.abs(G["g_q"]).max() + 1))
