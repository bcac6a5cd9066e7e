"""ctypes view of libshw.so (the C ABI declared in include/shw.h).

Argument marshalling only: every computation happens in the library's CUDA
kernels.  Loading fails loudly when the library has not been built; there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libshw.so")

SHW_OK, SHW_EINVAL, SHW_EUNSUPPORTED, SHW_ECUDA, SHW_ENOMEM, SHW_ETIMEOUT, SHW_EDEVICE, SHW_EBOUNDS = range(8)
MODES = {"mip": 0, "avg": 1, "composite": 2, "spectral": 3, "ratio": 4, "moment1": 5,
         "composite_spectral": 6, "mip_rgb": 7, "composite_rgb": 8, "ratio_mip": 9}
INTERP = {"nearest": 0, "trilinear": 1}
STORAGE = {"f32": 0, "bf16": 1, "f16": 2, "pair": 3, "bf16_pair": 4, "f16_pair": 5, "bf16_linear": 6,
           "f16_linear": 7, "bf16_linear_pair": 8, "f16_linear_pair": 9}
ABI_VERSION = 5
LUT_SIZE = 256
MAX_SMOOTH_RADIUS = 16
BRICK = 32
BRICK_STORED = 34


class Volume(C.Structure):
    _fields_ = [("data", C.c_void_p), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("storage", C.c_int32)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3), ("fwd", C.c_float * 3),
                ("tan_half_fovy", C.c_float), ("ortho_half_h", C.c_float), ("ortho", C.c_int32),
                ("width", C.c_int32), ("height", C.c_int32)]


class RenderParams(C.Structure):
    _fields_ = [("mode", C.c_int32), ("interp", C.c_int32), ("step", C.c_float), ("lo", C.c_float),
                ("hi", C.c_float), ("lut", C.c_void_p), ("opacity_scale", C.c_float),
                ("term_alpha", C.c_float), ("ratio_floor", C.c_float), ("ckpt_interval", C.c_int32),
                ("filter", C.c_int32), ("min_threshold", C.c_float), ("max_threshold", C.c_float),
                ("alpha_threshold", C.c_int32), ("smooth", C.c_int32), ("smooth_arm", C.c_int32),
                ("smooth_ntaps", C.c_int32), ("smooth_c0", C.c_float), ("smooth_offset", C.c_float * 4),
                ("smooth_weight", C.c_float * 4)]

FILTERS = {None: 0, "none": 0, "clip": 1, "scale": 2}
SMOOTH = {None: 0, "none": 0, "box": 1, "taps": 2}
MAX_SMOOTH_TAPS = 4


class BatchItem(C.Structure):
    _fields_ = [("vol", Volume), ("cam", Camera), ("out_rgba", C.c_void_p), ("mode", C.c_int32)]


class BatchInfo(C.Structure):
    _fields_ = [("n_items", C.c_int32), ("n_work", C.c_int32), ("tile", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("grid", C.c_int32), ("tuned", C.c_int32), ("brick", C.c_int32), ("n_candidates", C.c_int32),
                ("cand_tile", C.c_int32 * 16), ("cand_ctas_per_sm", C.c_int32 * 16), ("cand_brick", C.c_int32 * 16),
                ("tune_ms", C.c_float * 16), ("packed_bytes", C.c_int64)]


BATCH_NO_TUNE, BATCH_RETUNE = 1, 2
BATCH_PACK = {None: 0, "bf16": 4, "f16": 8}   # the plan rounds float32 items into its own 16-bit bricks
BATCH_BRICK = {None: 0, 16: 16, 32: 32}       # with a pack storage: fix the brick edge (else tuned)


class ShwError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        msg = lib().shw_status_string(self.status).decode()
        super().__init__(f"{what}: {msg} (status {self.status})" if what else msg)


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_vp, _i32, _f, _sz = C.c_void_p, C.c_int32, C.c_float, C.c_size_t
_P = C.POINTER
SIGNATURES = {
    "shw_abi_version": (_i32, []),
    "shw_status_string": (C.c_char_p, [_i32]),
    "shw_struct_size": (_sz, [_i32]),
    "shw_launch_count": (C.c_uint64, []),
    "shw_sync_status": (_i32, [_vp]),
    "shw_smooth": (_i32, [_vp, _vp, _i32, _i32, _i32, _f, _i32, _vp]),
    "shw_smooth_weights": (_i32, [_vp, _vp, _i32, _i32, _i32, _P(C.c_float), _i32, _vp]),
    "shw_smooth_zip": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _f, _i32, _vp]),
    "shw_bricked_bytes": (_sz, [_i32, _i32, _i32, _i32]),
    "shw_pack_bricks": (_i32, [_vp, _i32, _i32, _i32, _i32, _vp, _sz, _vp]),
    "shw_render": (_i32, [_P(Volume), _P(Volume), _P(Camera), _P(RenderParams), _vp, _vp, _vp, _vp, _vp, _sz,
                          _vp]),
    "shw_ckpt_bytes": (_sz, [_P(Volume), _P(Camera), _P(RenderParams)]),
    "shw_render_backward": (_i32, [_P(Volume), _P(Camera), _P(RenderParams), _vp, _vp, _sz, _vp, _vp, _vp, _vp]),
    "shw_batch_plan_create": (_i32, [_P(_vp), _P(BatchItem), _i32, _P(RenderParams), _i32, _vp]),
    "shw_render_batch": (_i32, [_vp, _vp]),
    "shw_batch_plan_info": (_i32, [_vp, _P(BatchInfo)]),
    "shw_batch_plan_destroy": (_i32, [_vp]),
    "shw_render_batch_noalloc": (_i32, [_P(BatchItem), _i32, _P(RenderParams), _vp]),
    "shw_set_debug_flags": (C.c_uint32, [C.c_uint32]),
    "shw_render_items": (_i32, [_P(BatchItem), _i32, _P(RenderParams), _vp]),
    "shw_linear_sampling_taps": (_i32, [_P(C.c_double), _i32, _P(C.c_double), _P(C.c_double), _P(C.c_double), _i32,
                                        _P(_i32)]),
    "shw_binomial_taps": (_i32, [_i32, _i32, _P(C.c_double), _P(C.c_double), _P(C.c_double), _i32, _P(_i32)]),
}
# test and diagnosis switches of shw_set_debug_flags
DEBUG = {"no_axis_sweep": 0x1, "smooth_plain": 0x2, "box_direct": 0x4, "no_staging": 0x8, "fault_alloc": 0x10,
         "fault_graph": 0x20, "fault_timeout": 0x40, "require_staging": 0x80}
NOALLOC_SCRATCH_BYTES = 8 << 20


def lib():
    """The loaded library.  Raises if libshw.so is missing (build it with
    ``python -m paper_1707_00442_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is not built: run `python -m paper_1707_00442_gb300.build` "
                                  "(the CUDA library is required; there is no CPU fallback)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            if L.shw_abi_version() != ABI_VERSION:
                raise ImportError("libshw.so ABI version mismatch: rebuild it")
            for which, st in enumerate((Volume, Camera, RenderParams, BatchItem, BatchInfo)):
                if L.shw_struct_size(which) != C.sizeof(st):
                    raise ImportError(f"libshw.so struct layout mismatch for {st.__name__}")
            _lib = L
    return _lib


def check(status: int, what: str = "") -> None:
    if status != SHW_OK:
        raise ShwError(status, what)
