"""Seeded synthetic scene inputs shared by the CUDA path's tests/bench and the oracle.

This package holds ONLY input construction: noise cubes with Gaussian sources,
camera frames (eye/right/up/forward vectors), and RGBA lookup tables.  It holds
none of the ray-casting, sampling, transfer-function or smoothing arithmetic;
those live separately in the CUDA library and in the oracle.
"""
from .cubes import (  # noqa: F401
    SEED_BASE,
    STANDIN_DIMS,
    Source,
    add_source,
    batch_dims,
    batch_subcube,
    diff_cube,
    draw_sources,
    paper_standin,
    paper_uniform_cube,
    ratio_cube,
    survey_cube,
    tiny_cube,
)
from .camera import Camera, ortho_axis_camera, orbit_camera  # noqa: F401
from .lut import linear_lut, perturbed_lut, ratio_lut  # noqa: F401
