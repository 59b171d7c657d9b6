"""FP64 oracle of the decode-side epilogues: the steps that turn a decoder's outputs
into march inputs, and their gradients.

TEST INFRASTRUCTURE: the oracle is never on the product path. Plain numpy, written
from the paper's definitions:
- opacity fade factor (Sec. 3.1.3, Eq. for W): W(x, y, z) = exp(-alpha (x^beta + y^beta
  + z^beta)) over normalised payload coordinates in [-1, 1]^3, multiplying opacity;
- a view's payload (Sec. 3.1.3): RGB from the view-conditioned colour decoder, opacity
  from the view-independent one, faded, interleaved as RGBA;
- rotation from an axis-angle (Rodrigues) vector (Sec. 3.1.2), as a unit quaternion;
- volume minimisation prior (Sec. 3.3): L_vol = lambda sum_i Prod(s_i) over the
  primitives' side lengths.
"""
from __future__ import annotations

import numpy as np


def fade_window(M: int, alpha: float = 8.0, beta: int = 8) -> np.ndarray:
    """W over the M^3 payload voxels, [z][y][x]; a voxel's normalised coordinate is
    2 i/(M - 1) - 1 per axis (voxel centres on the box corners and faces)."""
    u = 2.0 * np.arange(M, dtype=np.float64) / (M - 1) - 1.0
    p = u ** beta
    s = p[:, None, None] + p[None, :, None] + p[None, None, :]
    return np.exp(-alpha * s)


def fade_payload(payload, alpha: float = 8.0, beta: int = 8) -> np.ndarray:
    """payload [n][M][M][M][4] with the opacity (channel 3) multiplied by W (FP64)."""
    P = np.array(payload, dtype=np.float64)
    P[..., 3] *= fade_window(P.shape[1], alpha, beta)[None]
    return P


def assemble_payload(rgb, opacity, alpha: float = 8.0, beta: int = 8) -> np.ndarray:
    """[n][M][M][M][4] FP64: channels 0-2 the view's colour rgb [n][M][M][M][3],
    channel 3 the shared opacity [n][M][M][M] times W (no fade at alpha = 0)."""
    rgb = np.asarray(rgb, np.float64)
    op = np.asarray(opacity, np.float64)
    P = np.empty(rgb.shape[:-1] + (4,))
    P[..., :3] = rgb
    P[..., 3] = op * fade_window(rgb.shape[1], alpha, beta)[None]
    return P


def axis_angle_to_quat(r) -> np.ndarray:
    """q = (cos(th/2), sin(th/2) r/th), th = |r|; the identity at r = 0."""
    r = np.asarray(r, np.float64)
    th = np.linalg.norm(r, axis=-1)
    q = np.zeros(r.shape[:-1] + (4,))
    q[..., 0] = np.cos(th / 2)
    safe = np.where(th > 0, th, 1.0)
    f = np.where(th > 0, np.sin(th / 2) / safe, 0.5)
    q[..., 1:] = f[..., None] * r
    return q


def axis_angle_vjp(r, g_q) -> np.ndarray:
    """(dq/dr)^T g_q by differentiating axis_angle_to_quat: with f(th) = sin(th/2)/th,
    dq_w/dr = -(f/2) r and dq_v/dr = f I + (f'(th)/th) r r^T."""
    r = np.asarray(r, np.float64)
    g_q = np.asarray(g_q, np.float64)
    th = np.linalg.norm(r, axis=-1)
    safe = np.where(th > 0, th, 1.0)
    f = np.where(th > 0, np.sin(th / 2) / safe, 0.5)
    fp_over_th = np.where(th > 1e-4, (0.5 * safe * np.cos(safe / 2) - np.sin(safe / 2)) / safe ** 3,
                          -1.0 / 24.0 + th ** 2 / 960.0)
    dot = np.sum(g_q[..., 1:] * r, axis=-1)
    a = -0.5 * f * g_q[..., 0] + fp_over_th * dot
    return a[..., None] * r + f[..., None] * g_q[..., 1:]


def volume_prior(s, lam: float = 0.01):
    """(L_vol, dL_vol/ds) for half extents s [n][3]: side lengths are 2 s."""
    s = np.asarray(s, np.float64)
    side = 2.0 * s
    loss = lam * np.sum(np.prod(side, axis=1))
    g = np.empty_like(s)
    g[:, 0] = 2.0 * lam * side[:, 1] * side[:, 2]
    g[:, 1] = 2.0 * lam * side[:, 0] * side[:, 2]
    g[:, 2] = 2.0 * lam * side[:, 0] * side[:, 1]
    return loss, g
