"""Seeded synthetic stereo pairs shaped like the fast-bilateral-stereo workloads.

This package only produces inputs (images, ground-truth disparities,
occlusion masks and workload parameters).  It holds none of the matching
arithmetic, so both the CPU oracle and the CUDA path may use it.
"""

from .scenes import (  # noqa: F401
    WORKLOADS,
    Pair,
    make_workload,
    make_pair,
    shifted_texture_pair,
    constant_image,
    random_batch_specs,
    render_layers,
    regions,
)
