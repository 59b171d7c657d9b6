"""Pins of the decode-side epilogue oracle (oracle/decode.py) to facts outside it:
scipy's rotation-vector conversion, closed forms, symmetries and finite differences."""
import numpy as np
import pytest

from oracle import decode as D


def test_fade_window_closed_forms():
    M = 9  # odd: the centre voxel sits at (0, 0, 0)
    W = D.fade_window(M, 8.0, 8)
    assert W[4, 4, 4] == 1.0                              # W(0,0,0) = exp(0)
    assert np.isclose(W[0, 0, 0], np.exp(-24.0))          # a corner: x^8 = y^8 = z^8 = 1
    assert np.isclose(W[4, 4, 8], np.exp(-8.0))           # face centre (1, 0, 0)
    assert np.isclose(W[4, 4, 6], np.exp(-8.0 * 0.5 ** 8))  # x = 2*6/8 - 1 = 0.5
    # symmetric under each axis flip, and separable: W = w(x) w(y) w(z)
    assert np.array_equal(W, W[::-1]) and np.array_equal(W, W[:, ::-1]) and np.array_equal(W, W[:, :, ::-1])
    w1 = D.fade_window(M, 8.0, 8)[4, 4, :]
    assert np.allclose(W, w1[:, None, None] * w1[None, :, None] * w1[None, None, :], rtol=1e-14)
    # alpha = 0 or beta = 0 give constants
    assert np.all(D.fade_window(5, 0.0, 8) == 1.0)
    assert np.allclose(D.fade_window(5, 2.0, 0), np.exp(-6.0))


def test_fade_payload_touches_only_opacity():
    rng = np.random.default_rng(0)
    P = rng.uniform(0, 1, (3, 6, 6, 6, 4))
    F = D.fade_payload(P, 8.0, 8)
    assert np.array_equal(F[..., :3], P[..., :3])
    assert np.allclose(F[..., 3], P[..., 3] * D.fade_window(6, 8.0, 8)[None])
    assert np.all(F[..., 3] <= P[..., 3])


def test_axis_angle_matches_scipy():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(1)
    r = rng.standard_normal((200, 3)) * rng.uniform(0, 3.0, (200, 1))
    r[:3] = [[0, 0, 0], [1e-9, 0, 0], [0, 0, np.pi - 1e-6]]
    q = D.axis_angle_to_quat(r)
    ref = Rot.from_rotvec(r).as_quat()  # (x, y, z, w)
    ref = np.concatenate([ref[:, 3:], ref[:, :3]], axis=1)
    assert np.allclose(q, ref, atol=1e-12)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0)


def test_axis_angle_vjp_matches_finite_differences():
    rng = np.random.default_rng(2)
    r = rng.standard_normal((40, 3)) * rng.uniform(0, 3.0, (40, 1))
    r[0] = [0, 0, 0]
    r[1] = [2e-5, -1e-5, 3e-5]  # inside the series branch of the derivative
    g = rng.standard_normal((40, 4))
    v = D.axis_angle_vjp(r, g)
    h = 1e-6
    fd = np.zeros_like(r)
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd[:, j] = np.sum((D.axis_angle_to_quat(r + e) - D.axis_angle_to_quat(r - e)) * g, axis=1) / (2 * h)
    assert np.allclose(v, fd, atol=1e-8)


def test_volume_prior_closed_form_and_gradient():
    s = np.array([[0.5, 1.0, 2.0], [0.1, 0.2, 0.3]])
    loss, g = D.volume_prior(s, 0.01)
    # side lengths (1, 2, 4) and (0.2, 0.4, 0.6): volumes 8 and 0.048
    assert np.isclose(loss, 0.01 * (8.0 + 0.048))
    h = 1e-7
    for k in range(2):
        for j in range(3):
            sp, sm = s.copy(), s.copy()
            sp[k, j] += h
            sm[k, j] -= h
            fd = (D.volume_prior(sp, 0.01)[0] - D.volume_prior(sm, 0.01)[0]) / (2 * h)
            assert np.isclose(g[k, j], fd, rtol=1e-7)


def test_assemble_payload_interleaves_and_fades():
    rng = np.random.default_rng(3)
    rgb = rng.uniform(0, 1, (2, 5, 5, 5, 3))
    op = rng.uniform(0, 4, (2, 5, 5, 5))
    P = D.assemble_payload(rgb, op, 0.0, 8)  # no fade: plain interleaving
    assert P.shape == (2, 5, 5, 5, 4)
    assert np.array_equal(P[..., :3], rgb) and np.array_equal(P[..., 3], op)
    F = D.assemble_payload(rgb, op, 8.0, 8)
    assert np.array_equal(F[..., :3], rgb)
    assert F[0, 2, 2, 2, 3] == op[0, 2, 2, 2]                      # W = 1 at the centre
    assert np.isclose(F[1, 0, 0, 0, 3], op[1, 0, 0, 0] * np.exp(-24.0))  # a corner
    assert np.isclose(F[1, 2, 2, 4, 3], op[1, 2, 2, 4] * np.exp(-8.0))   # a face centre
