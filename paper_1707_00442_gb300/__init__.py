"""GB300-native spectral-cube ray caster (Vohl et al. 2017, "Real-time colouring
and filtering with graphics shaders"): a C-ABI CUDA library (libshw.so, sm_103a)
with this thin PyTorch binding.  See include/shw.h for the contract of each call.
"""
from .api import (  # noqa: F401
    BatchPlan,
    BrickVolume,
    ShwError,
    binomial_taps,
    bricked_bytes,
    ckpt_bytes,
    debug_flags,
    launch_count,
    linear_sampling_taps,
    pack_bricks,
    render,
    render_backward,
    smooth,
    smooth_weights,
    smooth_zip,
    sync_status,
)
from .autograd import composite_render  # noqa: F401
from ._lib import LIB_PATH, MODES, INTERP, STORAGE  # noqa: F401
