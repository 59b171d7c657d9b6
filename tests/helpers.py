"""Small test-only helpers: scene surgery and rotations through scipy (independent of
both the oracle and the CUDA path)."""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation

import synthetic


def rot_matrix(q_wxyz) -> np.ndarray:
    q = np.asarray(q_wxyz, np.float64)
    return Rotation.from_quat(q[..., [1, 2, 3, 0]]).as_matrix()


def quat_from_matrix(R) -> np.ndarray:
    x = Rotation.from_matrix(R).as_quat()
    return x[..., [3, 0, 1, 2]]


def single_box(M=4, alpha=1.0, rgb=(0.25, 0.5, 0.75), t=(0, 0, 0), q=(1, 0, 0, 0), s=(0.3, 0.3, 0.3)):
    payload = np.zeros((1, M, M, M, 4), np.float32)
    payload[..., :3] = np.asarray(rgb, np.float32)
    payload[..., 3] = alpha
    return synthetic.Scene(t=np.asarray([t], np.float32), q=np.asarray([q], np.float32),
                           s=np.asarray([s], np.float32), payload=payload, M=M)


def rays_from(o, d, t_near, t_far, dt, eps=0.0, bg=(0, 0, 0), width=0, height=0):
    o = np.ascontiguousarray(np.atleast_2d(np.asarray(o, np.float32)))
    d = np.ascontiguousarray(np.atleast_2d(np.asarray(d, np.float32)))
    if o.shape[0] == 1 and d.shape[0] > 1:
        o = np.ascontiguousarray(np.repeat(o, d.shape[0], 0))
    return synthetic.Rays(o=o, d=d, t_near=t_near, t_far=t_far, dt=dt, eps_early=eps, bg=tuple(bg),
                          width=width, height=height)


def concat_scenes(a, b):
    assert a.M == b.M
    return synthetic.Scene(t=np.concatenate([a.t, b.t]), q=np.concatenate([a.q, b.q]),
                           s=np.concatenate([a.s, b.s]), payload=np.concatenate([a.payload, b.payload]),
                           M=a.M)


def permute_scene(sc, perm):
    return synthetic.Scene(t=sc.t[perm].copy(), q=sc.q[perm].copy(), s=sc.s[perm].copy(),
                           payload=sc.payload[perm].copy(), M=sc.M)


def zero_boundary(sc):
    """Payload with every face voxel zeroed: the sampled field is then continuous across
    box faces (zero on both sides), so finite differences see no jumps there."""
    p = sc.payload.copy()
    p[:, 0] = 0
    p[:, -1] = 0
    p[:, :, 0] = 0
    p[:, :, -1] = 0
    p[:, :, :, 0] = 0
    p[:, :, :, -1] = 0
    return synthetic.Scene(t=sc.t, q=sc.q, s=sc.s, payload=p, M=sc.M)


def rays_from_matrix(m34, focal, width, height, t_near, t_far, dt):
    """Pinhole rays of a row-major 3x4 camera matrix [right down forward | eye] (the
    matrix a serving request carries), through pixel centres (col + 0.5, row + 0.5)
    about the image centre, computed in FP64 and stored FP32 (row-major pixels)."""
    m = np.asarray(m34, np.float64).reshape(3, 4)
    cols = (np.arange(width) + 0.5 - width / 2.0) / float(np.float32(focal))
    rows = (np.arange(height) + 0.5 - height / 2.0) / float(np.float32(focal))
    xx, yy = np.meshgrid(cols, rows)
    dc = np.stack([xx, yy, np.ones_like(xx)], axis=-1).reshape(-1, 3)
    d = dc @ m[:, :3].T
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(m[:, 3], d.shape)
    return rays_from(o, d, t_near, t_far, dt, width=width, height=height)
