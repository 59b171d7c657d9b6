"""CPU oracle of the MVP ray march (FP64, plain loops).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU baseline
leg of ``bench.py`` may import this package. The product package never imports it,
and it never imports the product package.
"""
from .oracle import (  # noqa: F401
    build,
    hit_lists,
    morton_keys,
    radix_tree,
    render,
    backward,
    rotations,
    rotations_f32spec,
    MODE_BRUTE,
    MODE_PRUNED,
    MEMBER_F64,
    MEMBER_F32,
    SEQUENTIAL,
    LITERAL,
)
