"""ctypes wrapper around ``mvp_oracle.c`` (see that file for the paper passages).

TEST INFRASTRUCTURE: the oracle is never on the product path.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mvp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

MODE_BRUTE = 0
MODE_PRUNED = 1
MEMBER_F64 = 0
MEMBER_F32 = 2
SEQUENTIAL = 4  # the saturating sample blended primitive by primitive in BVH order
LITERAL = 8  # background composite A I + (1 - A) B

_lib = None


def _lib_path() -> str:
    with open(_SRC, "rb") as f:
        h = hashlib.sha1(f.read()).hexdigest()[:12]
    return os.path.join(_BUILD, f"libmvp_oracle_{h}.so")


def build() -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction). Returns the .so path."""
    path = _lib_path()
    if not os.path.exists(path):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32, i64, f32 = ctypes.c_int, ctypes.c_int64, ctypes.c_float
    lib.orc_rotations.argtypes = [i32, P, P]
    lib.orc_rotations_f32spec.argtypes = [i32, P, P]
    lib.orc_hit_counts.argtypes = [i32, P, P, P, i64, P, P, f32, f32, i32, P]
    lib.orc_hit_fill.argtypes = [i32, P, P, P, i64, P, P, f32, f32, i32, P, P, P, P, P]
    lib.orc_morton_keys.argtypes = [i32, P, P, P]
    lib.orc_radix_tree.argtypes = [i32, P, P, P]
    lib.orc_render.argtypes = [i32, i32, P, P, P, P, i64, P, P, f32, f32, f32, f32, P, i32, i32, i32,
                               P, P, P, P, P, P, P]
    lib.orc_render.restype = i32
    lib.orc_backward.argtypes = [i32, i32, P, P, P, P, i64, P, P, f32, f32, f32, f32, P, i32, i32, i32,
                                 P, P, P, P, P]
    lib.orc_backward.restype = i32
    _lib = lib
    return lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def rotations(q) -> np.ndarray:
    q = _c(q, np.float32)
    out = np.zeros((q.shape[0], 3, 3), np.float64)
    _load().orc_rotations(q.shape[0], _p(q), _p(out))
    return out


def rotations_f32spec(q) -> np.ndarray:
    q = _c(q, np.float32)
    out = np.zeros((q.shape[0], 3, 3), np.float32)
    _load().orc_rotations_f32spec(q.shape[0], _p(q), _p(out))
    return out


def hit_lists(t, q, s, o, d, t_near, t_far, spec: str = "f32"):
    """Per-ray hit lists as CSR: (offs [R+1], ids, tin, tout, margin).

    spec "f32": the FP32 decision (fixed operation order); "f64": FP64 intervals,
    including near misses with tout - tin >= -1e-4 so grazing pairs can be told apart
    (margin = tout - tin)."""
    lib = _load()
    t, q, s = _c(t, np.float32), _c(q, np.float32), _c(s, np.float32)
    o, d = _c(o, np.float32), _c(d, np.float32)
    n, R = t.shape[0], o.shape[0]
    sp = 1 if spec == "f32" else 0
    counts = np.zeros(R, np.int64)
    lib.orc_hit_counts(n, _p(t), _p(q), _p(s), R, _p(o), _p(d), t_near, t_far, sp, _p(counts))
    offs = np.zeros(R + 1, np.int64)
    np.cumsum(counts, out=offs[1:])
    H = int(offs[-1])
    ids = np.zeros(H, np.int32)
    tin = np.zeros(H, np.float64)
    tout = np.zeros(H, np.float64)
    margin = np.zeros(H, np.float64)
    lib.orc_hit_fill(n, _p(t), _p(q), _p(s), R, _p(o), _p(d), t_near, t_far, sp, _p(offs), _p(ids),
                     _p(tin), _p(tout), _p(margin))
    return offs, ids, tin, tout, margin


def morton_keys(t):
    """(bounds [6] float32 = lo xyz, hi xyz; keys [N] uint64 = morton << 32 | k)."""
    t = _c(t, np.float32)
    n = t.shape[0]
    bounds = np.zeros(6, np.float32)
    keys = np.zeros(n, np.uint64)
    _load().orc_morton_keys(n, _p(t), _p(bounds), _p(keys))
    return bounds, keys


def radix_tree(sorted_keys):
    """Children (left, right) of the n-1 internal nodes; leaf j is node n-1+j."""
    k = _c(sorted_keys, np.uint64)
    n = k.shape[0]
    left = np.full(max(n - 1, 0), -1, np.int32)
    right = np.full(max(n - 1, 0), -1, np.int32)
    _load().orc_radix_tree(n, _p(k), _p(left), _p(right))
    return left, right


def _march_args(scene, rays, n_steps=None):
    t, q, s = _c(scene.t, np.float32), _c(scene.q, np.float32), _c(scene.s, np.float32)
    payload = _c(scene.payload, np.float32)
    o, d = _c(rays.o, np.float32), _c(rays.d, np.float32)
    bg = np.asarray(rays.bg, np.float32)
    ns = rays.n_steps if n_steps is None else n_steps
    return t, q, s, payload, o, d, bg, ns


def render(scene, rays, mode: int = MODE_PRUNED | MEMBER_F32, n_threads: int = 0):
    """FP64 render. Returns dict with rgba [R,4] float64, near_face [R] bool,
    n_eval [R] int64, i_last [R], i_clamp [R], beta [R] (the adjoint's clamp weight),
    clamp_k [R] (sequential rule: the primitive clamped at i_clamp, -1 if none)."""
    t, q, s, payload, o, d, bg, ns = _march_args(scene, rays)
    R = o.shape[0]
    out = np.zeros((R, 4), np.float64)
    nf = np.zeros(R, np.uint8)
    ne = np.zeros(R, np.int64)
    il = np.zeros(R, np.int32)
    ic = np.zeros(R, np.int32)
    be = np.zeros(R, np.float64)
    ck = np.zeros(R, np.int32)
    rc = _load().orc_render(t.shape[0], scene.M, _p(t), _p(q), _p(s), _p(payload), R, _p(o), _p(d),
                            rays.t_near, rays.t_far, rays.dt, rays.eps_early, _p(bg), ns, mode,
                            n_threads, _p(out), _p(nf), _p(ne), _p(il), _p(ic), _p(be), _p(ck))
    if rc != 0:
        raise ValueError("oracle render rejected its arguments")
    return {"rgba": out, "near_face": nf.astype(bool), "n_eval": ne, "i_last": il, "i_clamp": ic, "beta": be,
            "clamp_k": ck}


def backward(scene, rays, grad_out, mode: int = MODE_PRUNED | MEMBER_F32, n_threads: int = 0):
    """FP64 adjoint: dict of g_payload [N,M,M,M,4], g_t [N,3], g_q [N,4], g_s [N,3]."""
    t, q, s, payload, o, d, bg, ns = _march_args(scene, rays)
    R, n = o.shape[0], t.shape[0]
    go = _c(grad_out, np.float64).reshape(R, 4)
    gp = np.zeros(payload.shape, np.float64)
    gt = np.zeros((n, 3), np.float64)
    gq = np.zeros((n, 4), np.float64)
    gs = np.zeros((n, 3), np.float64)
    rc = _load().orc_backward(n, scene.M, _p(t), _p(q), _p(s), _p(payload), R, _p(o), _p(d),
                              rays.t_near, rays.t_far, rays.dt, rays.eps_early, _p(bg), ns, mode,
                              n_threads, _p(go), _p(gp), _p(gt), _p(gq), _p(gs))
    if rc != 0:
        raise ValueError("oracle backward rejected its arguments")
    return {"g_payload": gp, "g_t": gt, "g_q": gq, "g_s": gs}
