"""ctypes binding of ``include/mvp.h``: same names, argument marshalling only.

The shared library is compiled from ``csrc/`` for sm_103a by :mod:`.build`. There is
no fallback: if the library cannot be built or loaded, importing the functions
raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32, c_int64, c_float, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                                 ctypes.c_void_p, ctypes.c_size_t)

MVP_OK = 0
MVP_NOT_READY = 1
MVP_ERR_INVALID_ARG = -1
MVP_ERR_CUDA = -2
MVP_ERR_OOM = -3
MVP_ERR_CAPACITY = -4
MVP_ERR_TIMEOUT = -5
MVP_ERR_DEVICE = -6

MVP_F32, MVP_BF16, MVP_F16 = 0, 1, 2
MVP_BLEND_SEQUENTIAL = 1
MVP_COMPOSITE_LITERAL = 2


class mvp_prims(ctypes.Structure):
    _fields_ = [("n", c_int32), ("M", c_int32), ("dtype", c_int32), ("reserved", c_int32),
                ("t", c_void_p), ("q", c_void_p), ("s", c_void_p), ("payload", c_void_p)]


class mvp_rays(ctypes.Structure):
    _fields_ = [("n", c_int64), ("o", c_void_p), ("d", c_void_p), ("t_near", c_float), ("t_far", c_float),
                ("dt", c_float), ("eps_early", c_float), ("bg", c_float * 3), ("width", c_int32),
                ("height", c_int32), ("flags", c_int32)]


class mvp_request(ctypes.Structure):
    _fields_ = [("avatar", c_int32), ("width", c_int32), ("height", c_int32), ("focal", c_float),
                ("c2w", c_float * 12), ("t_near", c_float), ("t_far", c_float), ("dt", c_float),
                ("eps_early", c_float), ("bg", c_float * 3), ("views", c_int32), ("c2w_right", c_float * 12),
                ("payload", c_void_p)]


class mvp_serve_info(ctypes.Structure):
    _fields_ = [("pending", c_int64), ("in_flight", c_int64), ("max_in_flight", c_int64), ("completed", c_int64),
                ("resident_bytes", c_int64), ("in_flight_bytes", c_int64), ("grid_blocks", c_int32),
                ("avatars", c_int32), ("device_status", c_int32), ("reserved", c_int32), ("batches", c_int64),
                ("cancelled", c_int64)]


class MVPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} [{status}]")
        self.status = status


_LIB = None

# (name, restype, argtypes) for every function of include/mvp.h
_SIGS = [
    ("mvp_version", ctypes.c_char_p, []),
    ("mvp_status_string", ctypes.c_char_p, [c_int32]),
    ("mvp_last_error", ctypes.c_char_p, []),
    ("mvp_num_steps", c_int64, [c_float, c_float, c_float]),
    ("mvp_ctx_create", c_int32, [c_int32, ctypes.POINTER(c_void_p)]),
    ("mvp_ctx_destroy", None, [c_void_p]),
    ("mvp_ctx_sync", c_int32, [c_void_p, c_void_p]),
    ("mvp_bvh_create", c_int32, [c_void_p, ctypes.POINTER(c_void_p)]),
    ("mvp_bvh_destroy", None, [c_void_p]),
    ("mvp_build_bvh", c_int32, [c_void_p, ctypes.POINTER(mvp_prims), c_void_p, c_void_p]),
    ("mvp_bvh_size", c_int32, [c_void_p]),
    ("mvp_bvh_export", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("mvp_hitlists", c_int32, [c_void_p, ctypes.POINTER(mvp_prims), c_void_p, ctypes.POINTER(mvp_rays), c_void_p,
                               c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(c_int64), c_void_p]),
    ("mvp_saved_bytes", c_size_t, [c_int64]),
    ("mvp_raymarch_fwd", c_int32, [c_void_p, ctypes.POINTER(mvp_prims), c_void_p, ctypes.POINTER(mvp_rays),
                                   c_void_p, c_void_p, c_void_p]),
    ("mvp_raymarch_count", c_int32, [c_void_p, ctypes.POINTER(mvp_prims), c_void_p, ctypes.POINTER(mvp_rays),
                                     c_void_p, c_void_p]),
    ("mvp_raymarch_bwd", c_int32, [c_void_p, ctypes.POINTER(mvp_prims), c_void_p, ctypes.POINTER(mvp_rays),
                                   c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("mvp_pack_payload", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_void_p]),
    ("mvp_camera_rays", c_int32, [c_void_p, ctypes.POINTER(c_float), c_float, c_int32, c_int32, c_void_p,
                                  c_void_p, c_void_p]),
    ("mvp_serve_create", c_int32, [c_void_p, c_size_t, c_int32, c_size_t, ctypes.POINTER(c_void_p)]),
    ("mvp_serve_destroy", None, [c_void_p]),
    ("mvp_serve_register_avatar", c_int32, [c_void_p, ctypes.POINTER(mvp_prims), ctypes.POINTER(c_int32)]),
    ("mvp_serve_submit", c_int32, [c_void_p, ctypes.POINTER(mvp_request), ctypes.POINTER(ctypes.c_uint64)]),
    ("mvp_serve_poll", c_int32, [c_void_p, ctypes.c_uint64, c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("mvp_serve_cancel", c_int32, [c_void_p, ctypes.c_uint64]),
    ("mvp_serve_wait", c_int32, [c_void_p, ctypes.c_uint64, ctypes.c_double, c_void_p,
                                 ctypes.POINTER(ctypes.c_double)]),
    ("mvp_serve_stats", c_int32, [c_void_p, ctypes.POINTER(mvp_serve_info)]),
    ("mvp_raymarch_fwd_static", c_int32, [ctypes.POINTER(mvp_prims), ctypes.POINTER(mvp_rays), c_void_p, c_void_p,
                                          c_void_p]),
    ("mvp_fade_payload", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_float, c_int32,
                                   c_void_p]),
    ("mvp_assemble_payload", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_float,
                                       c_int32, c_void_p]),
    ("mvp_bounds_checked", c_int32, []),
    ("mvp_ctx_set_tile_schedule", c_int32, [c_void_p, c_int32]),
    ("mvp_ctx_set_bwd_group_bytes", c_int32, [c_void_p, c_int64]),
    ("mvp_axis_angle_to_quat", c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    ("mvp_axis_angle_backward", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    ("mvp_volume_prior", c_int32, [c_void_p, c_void_p, c_int32, c_float, c_void_p, c_void_p, c_void_p]),
    ("mvp_gather_probe", c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p,
                                   c_void_p, ctypes.POINTER(c_int64), c_void_p]),
]


def library_path() -> str:
    """The library to load: the checked build (device-side bounds checks) when the
    environment sets MVP_CHECK_BOUNDS=1, else the release build."""
    return _build.build(checked=os.environ.get("MVP_CHECK_BOUNDS") == "1")


def lib():
    """Load (building first if needed) libmvp.so; raises if that is impossible."""
    global _LIB
    if _LIB is None:
        path = library_path()
        L = ctypes.CDLL(path)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def check(status: int, what: str = "") -> int:
    """Raise MVPError for a negative status (with mvp_last_error's message)."""
    if status < 0:
        L = lib()
        msg = L.mvp_last_error().decode()
        name = L.mvp_status_string(status).decode()
        raise MVPError(status, f"{what}: {name}: {msg}")
    return status


def __getattr__(name):
    # mvp_* functions resolve to the loaded library's symbols
    if name.startswith("mvp_"):
        return getattr(lib(), name)
    raise AttributeError(name)


def loaded_path() -> str | None:
    return None if _LIB is None else os.path.realpath(_LIB._name)
