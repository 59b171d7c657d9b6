"""Seeded scenes, cameras and rays shaped like the paper's captures.

The paper's data (about 100 cameras on a 1.2 m sphere, 667x1024 images, trained
decoders producing primitives; Sec. 4.1) is not available, so every input here is
synthetic and drawn from ``numpy.random.default_rng(seed)``.

Conventions shared by every consumer of these arrays:

* Primitive k: centre ``t[k]`` (3), quaternion ``q[k]`` = (w, x, y, z) (4), half
  extents ``s[k]`` (3), payload ``payload[k, z, y, x, c]`` with c = (R, G, B, alpha)
  and x the fastest axis (Sec. 3.1.2 describes the payload as a 4 x M^3 voxel grid).
* Rays: ``o[r]``, ``d[r]`` float32, ``d`` unit length, row-major pixel order
  r = row * width + col for camera rays.
* Pinhole camera: camera axes right / down / forward, pixel centres at
  (col + 0.5, row + 0.5), principal point at the image centre.

Opacity values follow alpha = softplus(N(0, 1)) * 4 with a seeded fraction of voxels
set to zero, RGB ~ U[0, 1]. For the differentiation workload the alpha channel is
additionally shaped by the window exp(-8 (x^8 + y^8 + z^8)) over normalised voxel
coordinates (the opacity fade of Sec. 3.1.3, Eq. 1), which the paper applies to
decoder output upstream of the march.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Scene:
    t: np.ndarray  # [N, 3] float32 centres
    q: np.ndarray  # [N, 4] float32 quaternions (w, x, y, z)
    s: np.ndarray  # [N, 3] float32 half extents
    payload: np.ndarray  # [N, M, M, M, 4] float32, x fastest, RGBA last
    M: int

    @property
    def n(self) -> int:
        return int(self.t.shape[0])


@dataclass
class Camera:
    eye: np.ndarray  # [3] float64
    c2w: np.ndarray  # [3, 3] float64, columns = right, down, forward
    focal: float
    width: int
    height: int

    def matrix34(self) -> np.ndarray:
        """Camera-to-world as a row-major 3x4 float32 matrix [right down forward eye]."""
        m = np.zeros((3, 4), np.float64)
        m[:, :3] = self.c2w
        m[:, 3] = self.eye
        return m.astype(np.float32)


@dataclass
class Rays:
    o: np.ndarray  # [R, 3] float32
    d: np.ndarray  # [R, 3] float32, unit
    t_near: float
    t_far: float
    dt: float
    eps_early: float = 0.0
    bg: tuple = (0.0, 0.0, 0.0)
    width: int = 0  # 2-D tiling hint (0 = 1-D ray list)
    height: int = 0
    cameras: list = field(default_factory=list)

    @property
    def n(self) -> int:
        return int(self.o.shape[0])

    @property
    def n_steps(self) -> int:
        """Number of quadrature samples t_i = t_near + i*dt, i in [0, n_steps): the samples
        in [t_near, t_far), computed in double from the float32 values, where a sample
        within 1e-4*dt of t_far is not counted (so 4/0.01f gives 400, not 401)."""
        x = (float(np.float32(self.t_far)) - float(np.float32(self.t_near))) / float(np.float32(self.dt))
        return max(0, int(math.ceil(x - 1e-4)))


def random_unit_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _softplus(x: np.ndarray) -> np.ndarray:
    return np.logaddexp(np.float32(0.0), x).astype(np.float32)


def make_payload(rng: np.random.Generator, n: int, M: int, empty_frac: float,
                 fade: bool = False) -> np.ndarray:
    """[n, M, M, M, 4] float32 RGBA payload: RGB ~ U[0,1], alpha = softplus(N(0,1))*4,
    a fraction ``empty_frac`` of voxels (all four channels) set to zero."""
    shape = (n, M, M, M)
    out = np.empty(shape + (4,), np.float32)
    out[..., :3] = rng.random(shape + (3,), dtype=np.float32)
    out[..., 3] = _softplus(rng.standard_normal(shape, dtype=np.float32)) * np.float32(4.0)
    if empty_frac > 0:
        empty = rng.random(shape, dtype=np.float32) < np.float32(empty_frac)
        out[empty] = 0.0
    if fade:
        c = np.linspace(-1.0, 1.0, M)
        w = np.exp(-8.0 * (c[:, None, None] ** 8 + c[None, :, None] ** 8 + c[None, None, :] ** 8))
        out[..., 3] *= w.astype(np.float32)[None]
    return out


def view_colors(scene: Scene, view, seed: int = 0, strength: float = 0.5, power: int = 8) -> np.ndarray:
    """Stand-in for the view-conditioned colour decoder's output (the paper's colour
    decoder takes an object-centric view vector; its weights are not available):
    [N, M, M, M, 3] float32 = the scene's RGB plus a seeded per-voxel highlight
    strength * max(0, n . v)^power, clipped to [0, 1], with n a seeded unit vector per
    voxel (the same for every view) and v the unit view vector."""
    v = np.asarray(view, np.float32)
    v = v / np.linalg.norm(v)
    rng = np.random.default_rng(1000 + seed)
    shape = scene.payload.shape[:-1]
    nrm = rng.standard_normal(shape + (3,), dtype=np.float32)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    lobe = np.maximum(nrm @ v, 0.0) ** power
    rgb = scene.payload[..., :3] + np.float32(strength) * lobe[..., None]
    return np.clip(rgb, 0.0, 1.0).astype(np.float32)


def make_scene(n: int, M: int, seed: int, layout: str = "shell",
               s_range=(0.04, 0.08), s_const: float | None = None,
               empty_frac: float = 0.6, fade: bool = False,
               radii=(1.0, 1.2, 0.9), jitter: float = 0.02) -> Scene:
    """Seeded primitive set.

    layout "sphere": centres uniform on the unit sphere.
    layout "shell": centres on an ellipsoid shell with the given radii plus N(0, jitter^2)
    per-axis jitter. Half extents are ``s_const`` on every axis if given, else U[s_range]
    per axis.
    """
    rng = np.random.default_rng(seed)
    if layout == "sphere":
        t = _unit_vectors(rng, n)
    elif layout == "shell":
        t = _unit_vectors(rng, n) * np.asarray(radii)[None, :]
        t = t + rng.normal(0.0, jitter, size=(n, 3))
    else:
        raise ValueError(layout)
    q = random_unit_quaternions(rng, n)
    if s_const is not None:
        s = np.full((n, 3), s_const, np.float64)
    else:
        s = rng.uniform(s_range[0], s_range[1], size=(n, 3))
    payload = make_payload(rng, n, M, empty_frac, fade)
    return Scene(t=t.astype(np.float32), q=q, s=s.astype(np.float32), payload=payload, M=M)


def look_at_camera(eye, width: int, height: int, focal: float, target=(0.0, 0.0, 0.0)) -> Camera:
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 1.0, 0.0])
    if abs(float(fwd @ up)) > 0.99:
        up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    return Camera(eye=eye, c2w=np.stack([right, down, fwd], axis=1), focal=float(focal),
                  width=int(width), height=int(height))


def camera_rays(cam: Camera) -> tuple[np.ndarray, np.ndarray]:
    """Pinhole rays through pixel centres, row-major; computed in float64, stored float32."""
    cols = (np.arange(cam.width) + 0.5 - cam.width / 2.0) / cam.focal
    rows = (np.arange(cam.height) + 0.5 - cam.height / 2.0) / cam.focal
    xx, yy = np.meshgrid(cols, rows)
    dc = np.stack([xx, yy, np.ones_like(xx)], axis=-1).reshape(-1, 3)
    d = dc @ cam.c2w.T
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(cam.eye, d.shape)
    return np.ascontiguousarray(o, np.float32), np.ascontiguousarray(d, np.float32)


def random_camera(rng: np.random.Generator, radius: float, width: int, height: int,
                  focal: float) -> Camera:
    return look_at_camera(_unit_vectors(rng, 1)[0] * radius, width, height, focal)


def make_rays(cams: list[Camera], t_near: float, t_far: float, dt: float,
              eps_early: float = 0.0, bg=(0.0, 0.0, 0.0)) -> Rays:
    os_, ds_ = zip(*[camera_rays(c) for c in cams])
    one = len(cams) == 1
    return Rays(o=np.concatenate(os_), d=np.concatenate(ds_), t_near=t_near, t_far=t_far,
                dt=dt, eps_early=eps_early, bg=tuple(bg),
                width=cams[0].width if one else 0, height=cams[0].height if one else 0,
                cameras=list(cams))


def make_target(seed: int, width: int, height: int, n_images: int = 1) -> np.ndarray:
    """Seeded smooth RGB target image(s) in [0, 1]: a coarse random grid upsampled
    bilinearly. Shape [n_images * height * width, 3] float32, row-major per image."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_images):
        g = rng.random((9, 9, 3))
        ys = np.linspace(0, 8, height)
        xs = np.linspace(0, 8, width)
        y0 = np.minimum(ys.astype(int), 7)
        x0 = np.minimum(xs.astype(int), 7)
        fy = (ys - y0)[:, None, None]
        fx = (xs - x0)[None, :, None]
        a = g[y0][:, x0] * (1 - fx) + g[y0][:, x0 + 1] * fx
        b = g[y0 + 1][:, x0] * (1 - fx) + g[y0 + 1][:, x0 + 1] * fx
        out.append((a * (1 - fy) + b * fy).reshape(-1, 3))
    return np.concatenate(out).astype(np.float32)


def _shell_scale(n: int) -> tuple[float, float]:
    # Keep the shell's area coverage (sum of projected box areas) that of 4096 boxes
    # with half extents U[0.04, 0.08]: s scales with sqrt(4096 / n).
    f = math.sqrt(4096.0 / n)
    return (0.04 * f, 0.08 * f)


def make_config(name: str, seed: int = 0):
    """Return (scene, rays, extras) for a named workload; see CONFIGS."""
    spec = CONFIGS[name]
    return spec(seed)


def _c0(seed):
    scene = make_scene(8, 8, seed, layout="sphere", s_const=0.3, empty_frac=0.5)
    cam = random_camera(np.random.default_rng(seed + 1000), 3.0, 64, 64, 64.0)
    return scene, make_rays([cam], 1.0, 5.0, 0.01), {}


def _c1_factory(n, M, width=667, height=1024, focal=1024.0, dt=0.005):
    def f(seed):
        scene = make_scene(n, M, seed, layout="shell", s_range=_shell_scale(n), empty_frac=0.6)
        cam = random_camera(np.random.default_rng(seed + 1000), 3.0, width, height, focal)
        return scene, make_rays([cam], 1.0, 5.0, dt), {}
    return f


def _c3_factory(n=512, M=32, width=512, height=512, n_cams=4, dt=0.005):
    def f(seed):
        scene = make_scene(n, M, seed, layout="shell", s_range=_shell_scale(n), empty_frac=0.6,
                           fade=True)
        rng = np.random.default_rng(seed + 1000)
        cams = [random_camera(rng, 3.0, width, height, float(width)) for _ in range(n_cams)]
        rays = make_rays(cams, 1.0, 5.0, dt)
        target = make_target(seed + 2000, width, height, n_cams)
        return scene, rays, {"target": target}
    return f


# Serving avatars: (primitives, payload edge, seed offset); payloads are stored BF16.
AVATARS = [(512, 32, 0), (1024, 24, 0), (2048, 20, 0), (4096, 16, 0), (8192, 12, 0),
           (16384, 10, 0), (32768, 8, 0), (4096, 16, 1)]

SERVE_RESOLUTIONS = [(256, 256), (512, 512), (667, 1024)]  # (width, height)


def make_avatar(index: int, seed: int = 0, scale_down: int = 1) -> Scene:
    n, M, off = AVATARS[index]
    n = max(1, n // scale_down)
    return make_scene(n, M, seed * 100 + index * 7 + off, layout="shell",
                      s_range=_shell_scale(n), empty_frac=0.6)


CONFIGS = {
    # 8 primitives of 8^3, 64x64 image: the oracle runs in seconds.
    "tiny_8x8^3_64x64": _c0,
    # Paper-scale forward: 4096 primitives of 16^3 (about 256^3 voxels), 667x1024 image.
    "paper_4096x16^3_667x1024": _c1_factory(4096, 16),
    "sweep_512x32^3_667x1024": _c1_factory(512, 32),
    "sweep_32768x8^3_667x1024": _c1_factory(32768, 8),
    # Step-size sweep of the paper-scale frame (render time grows as 1/dt).
    "paper_4096x16^3_667x1024_dt0.01": _c1_factory(4096, 16, dt=0.01),
    "paper_4096x16^3_667x1024_dt0.0025": _c1_factory(4096, 16, dt=0.0025),
    # Reduced shapes of the same recipe, for parity tests that the oracle finishes quickly.
    "small_512x8^3_96x128": _c1_factory(512, 8, width=96, height=128, focal=128.0),
    "small_4096x16^3_83x128": _c1_factory(4096, 16, width=83, height=128, focal=128.0),
    # Differentiation: 512 primitives of 32^3 with the opacity window, 4 cameras of 512x512.
    "diff_512x32^3_4x512x512": _c3_factory(),
    "diff_small_64x8^3_2x48x40": _c3_factory(n=64, M=8, width=48, height=40, n_cams=2, dt=0.01),
}
