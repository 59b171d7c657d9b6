"""Seeded synthetic inputs for the MVP ray-march path.

This package draws random numbers and lays them out as primitives, payloads and
camera rays. It contains none of the method's own arithmetic (no rotation from a
quaternion, no ray/box test, no sampling or compositing), so the CUDA path and the
CPU oracle can both consume its arrays without sharing any of the method's code.
"""
from .scenes import (  # noqa: F401
    Camera,
    Rays,
    Scene,
    AVATARS,
    CONFIGS,
    SERVE_RESOLUTIONS,
    camera_rays,
    make_avatar,
    make_payload,
    make_rays,
    random_camera,
    look_at_camera,
    make_config,
    make_scene,
    make_target,
    random_unit_quaternions,
    view_colors,
)
