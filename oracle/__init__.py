"""FP64 CPU oracle of the spectral-cube ray caster -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its Python
binding) never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C99, double precision, OpenMP over
rays).  This module compiles it with gcc and wraps it for numpy: every input is
promoted exactly to float64 before the call.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODES = {"mip": 0, "avg": 1, "composite": 2, "spectral": 3, "ratio": 4, "moment1": 5,
         "composite_spectral": 6, "mip_rgb": 7, "composite_rgb": 8, "ratio_mip": 9}
INTERP = {"nearest": 0, "trilinear": 1}
FRAG_COUNT, FRAG_ROUND, FRAG_RATIO, FRAG_EXIT, FRAG_TIE = 1, 2, 4, 8, 16


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP, no -ffast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            dp, ip, lp, ucp, fp = (C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_long),
                                   C.POINTER(C.c_ubyte), C.POINTER(C.c_float))
            L.oracle_render.argtypes = [dp, dp, C.c_int, C.c_int, C.c_int, dp, C.c_int, C.c_int, C.c_int,
                                        C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, dp,
                                        C.c_double, C.c_double, C.c_double, lp, C.c_long, C.c_double,
                                        C.c_double, C.c_double, dp, dp, ip, ip, ucp]
            L.oracle_render2.argtypes = L.oracle_render.argtypes + [C.c_int, C.c_double, C.c_double, C.c_int]
            L.oracle_fetch_counter.argtypes = [C.c_int]
            L.oracle_fetches.restype = C.c_longlong
            L.oracle_render3.argtypes = L.oracle_render2.argtypes + [C.c_int, C.c_int, C.c_int, C.c_double,
                                                                     dp, dp]
            L.oracle_count_samples.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_int, C.c_int, C.c_int,
                                               C.c_double, ip]
            L.oracle_count_samples.restype = C.c_longlong
            L.oracle_ray_trace.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, C.c_int, C.c_int, C.c_int,
                                           C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, dp, dp]
            L.oracle_sample_points.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, dp, C.c_long, dp]
            L.oracle_gauss_weights.argtypes = [C.c_double, C.c_int, dp]
            L.oracle_binomial_weights.argtypes = [C.c_int, dp]
            L.oracle_linear_sampling_merge.argtypes = [dp, C.c_int, dp, dp]
            L.oracle_smooth_separable.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, C.c_int, dp]
            L.oracle_smooth_points.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, C.c_int, lp, C.c_long, dp]
            L.oracle_round_bf16.argtypes = [fp, C.c_long, fp]
            L.oracle_round_f16.argtypes = [fp, C.c_long, fp]
            L.oracle_render_grad.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, C.c_int, C.c_int, C.c_int,
                                             C.c_int, C.c_double, C.c_double, C.c_double, dp, C.c_double,
                                             C.c_double, dp, dp, dp, dp, dp]
            _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(C.POINTER(t))


def _cam_args(cam):
    return _d(cam.vec14()), int(bool(cam.ortho)), int(cam.width), int(cam.height)


FILTERS = {None: 0, "none": 0, "clip": 1, "scale": 2}
SMOOTH = {None: 0, "none": 0, "box": 1, "taps": 2}


def render(cube, cam, mode, *, interp="trilinear", step=0.5, lo=-3.0, hi=8.0, lut=None,
           opacity_scale=1.0, term_alpha=0.99, ratio_floor=0.0, cube2=None, pixels=None,
           eps_pos=0.0, eps_val=0.0, eps_exit=None, filter=None, min_threshold=0.0, max_threshold=0.0,
           alpha_threshold=False, smooth=None, smooth_arm=0, smooth_taps=None):
    """Render with the FP64 oracle.  Returns dict(rgba, scalar, index, nsamples, fragile).

    ``filter``: None, "clip" (Algorithm 10) or "scale" (Algorithm 11) with ``min_threshold`` /
    ``max_threshold``; ``alpha_threshold``: spectral / first-moment alpha 0 up to
    min_threshold, 1 above.

    ``smooth``: None, "box" (Algorithm 8, ``smooth_arm`` neighbours each side along the ray)
    or "taps" (Algorithm 9 per data axis, chained x, y, z) with ``smooth_taps`` =
    (c0, offsets, weights).

    ``pixels``: optional array of row-major pixel ids; outputs then follow that list.
    ``eps_pos`` / ``eps_val`` / ``eps_exit``: margins (voxels / values / opacity) within which a
    discrete decision of a ray is reported as fragile (diagnostic only).  eps_exit defaults to
    eps_val / 50.
    """
    if eps_exit is None:
        eps_exit = eps_val / 50.0
    L = lib()
    nz, ny, nx = cube.shape
    cubed = _d(cube)
    cube2d = _d(cube2) if cube2 is not None else None
    c14, ortho, W, H = _cam_args(cam)
    lutd = _d(lut).reshape(256, 4)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
    n = W * H if pix is None else len(pix)
    rgba = np.zeros((n, 4)); scal = np.zeros(n)
    idx = np.zeros(n, np.int32); ns = np.zeros(n, np.int32); fr = np.zeros(n, np.uint8)
    kind = SMOOTH[smooth]
    c0, toff, tw = 1.0, None, None
    if kind == 2:
        c0 = float(smooth_taps[0])
        toff = _d(np.asarray(smooth_taps[1], dtype=np.float64).ravel())
        tw = _d(np.asarray(smooth_taps[2], dtype=np.float64).ravel())
        if len(toff) != len(tw):
            raise ValueError("smooth_taps: offsets and weights differ in length")
    ntap = 0 if toff is None else len(toff)
    rc = L.oracle_render3(_ptr(cubed, C.c_double), _ptr(cube2d, C.c_double), nx, ny, nz,
                         _ptr(c14, C.c_double), ortho, W, H, MODES[mode], INTERP[interp],
                         float(step), float(lo), float(hi), _ptr(lutd, C.c_double),
                         float(opacity_scale), float(term_alpha), float(ratio_floor),
                         _ptr(pix, C.c_long), n, float(eps_pos), float(eps_val), float(eps_exit),
                         _ptr(rgba, C.c_double), _ptr(scal, C.c_double), _ptr(idx, C.c_int),
                         _ptr(ns, C.c_int), _ptr(fr, C.c_ubyte), FILTERS[filter], float(min_threshold),
                         float(max_threshold), int(bool(alpha_threshold)), kind, int(smooth_arm), ntap, c0,
                         _ptr(toff, C.c_double), _ptr(tw, C.c_double))
    if rc != 0:
        raise ValueError("oracle_render rejected its arguments")
    if pix is None:
        rgba, scal, idx, ns, fr = (rgba.reshape(H, W, 4), scal.reshape(H, W), idx.reshape(H, W),
                                   ns.reshape(H, W), fr.reshape(H, W))
    return {"rgba": rgba, "scalar": scal, "index": idx, "nsamples": ns, "fragile": fr}


def count_samples(dims, cam, step=0.5):
    """(total, per-ray N) of Algorithm 1's loop bound for every pixel."""
    L = lib()
    nx, ny, nz = dims
    c14, ortho, W, H = _cam_args(cam)
    out = np.zeros(W * H, np.int32)
    tot = L.oracle_count_samples(nx, ny, nz, _ptr(c14, C.c_double), ortho, W, H, float(step),
                                 _ptr(out, C.c_int))
    return int(tot), out.reshape(H, W)


def ray_trace(cube, cam, px, py, *, interp="trilinear", step=0.5, maxn=1 << 16):
    """Positions [N,3] and fetched values [N] of one ray's samples."""
    L = lib()
    nz, ny, nx = cube.shape
    c14, ortho, W, H = _cam_args(cam)
    pos = np.zeros((maxn, 3)); val = np.zeros(maxn)
    cubed = _d(cube)
    N = L.oracle_ray_trace(_ptr(cubed, C.c_double), nx, ny, nz, _ptr(c14, C.c_double), ortho, W, H,
                           INTERP[interp], float(step), int(px), int(py), maxn,
                           _ptr(pos, C.c_double), _ptr(val, C.c_double))
    N = min(N, maxn)
    return pos[:N], val[:N]


def sample_points(cube, pts, interp="trilinear"):
    """Algorithm 1's fetch at the given points [n, 3] (x, y, z in index space)."""
    nz, ny, nx = cube.shape
    cubed = _d(cube); P = _d(pts).reshape(-1, 3)
    out = np.zeros(len(P))
    lib().oracle_sample_points(_ptr(cubed, C.c_double), nx, ny, nz, INTERP[interp],
                               _ptr(P, C.c_double), len(P), _ptr(out, C.c_double))
    return out


def gauss_weights(sigma, r):
    w = np.zeros(2 * r + 1)
    lib().oracle_gauss_weights(float(sigma), int(r), _ptr(w, C.c_double))
    return w


def binomial_weights(n):
    w = np.zeros(n + 1)
    lib().oracle_binomial_weights(int(n), _ptr(w, C.c_double))
    return w


def linear_sampling_merge(w):
    w = _d(w)
    r = (len(w) - 1) // 2
    off = np.zeros(r + 2); wt = np.zeros(r + 2)
    m = lib().oracle_linear_sampling_merge(_ptr(w, C.c_double), r, _ptr(off, C.c_double),
                                           _ptr(wt, C.c_double))
    return off[:m + 1], wt[:m + 1]


def count_fetches(fn):
    """Run fn() with the oracle's fetch counter on; returns (fn's result, cube fetches made)."""
    L = lib()
    L.oracle_fetch_counter(1)
    try:
        out = fn()
        return out, int(L.oracle_fetches())
    finally:
        L.oracle_fetch_counter(0)


def smooth(cube, w):
    """Separable clamp-to-edge convolution with the 1-D kernel w on x, y, z in turn."""
    nz, ny, nx = cube.shape
    ind = _d(cube); w = _d(w); r = (len(w) - 1) // 2
    out = np.zeros_like(ind)
    if lib().oracle_smooth_separable(_ptr(ind, C.c_double), nx, ny, nz, _ptr(w, C.c_double), r,
                                     _ptr(out, C.c_double)) != 0:
        raise MemoryError("oracle_smooth_separable")
    return out


def smooth_points(cube, w, vox_ids):
    """The 3-D convolution as a direct triple sum, at the listed flat voxel ids only."""
    nz, ny, nx = cube.shape
    ind = _d(cube); w = _d(w); r = (len(w) - 1) // 2
    ids = np.ascontiguousarray(vox_ids, dtype=np.int64)
    out = np.zeros(len(ids))
    lib().oracle_smooth_points(_ptr(ind, C.c_double), nx, ny, nz, _ptr(w, C.c_double), r,
                               _ptr(ids, C.c_long), len(ids), _ptr(out, C.c_double))
    return out


def round_bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty_like(a)
    lib().oracle_round_bf16(_ptr(a, C.c_float), a.size, _ptr(out, C.c_float))
    return out


def round_f16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty_like(a)
    lib().oracle_round_f16(_ptr(a, C.c_float), a.size, _ptr(out, C.c_float))
    return out


def render_grad(cube, cam, grad_rgba, *, interp="trilinear", step=0.5, lo=-3.0, hi=8.0, lut=None,
                opacity_scale=1.0, term_alpha=0.99):
    """Reverse-mode gradient of the compositing render.  Returns (rgba, g_vol, g_lut, g_s)."""
    L = lib()
    nz, ny, nx = cube.shape
    cubed = _d(cube)
    c14, ortho, W, H = _cam_args(cam)
    lutd = _d(lut).reshape(256, 4)
    g = _d(grad_rgba).reshape(H * W * 4)
    rgba = np.zeros((H * W, 4)); gv = np.zeros_like(cubed); gl = np.zeros((256, 4)); gs = np.zeros(1)
    L.oracle_render_grad(_ptr(cubed, C.c_double), nx, ny, nz, _ptr(c14, C.c_double), ortho, W, H,
                         INTERP[interp], float(step), float(lo), float(hi), _ptr(lutd, C.c_double),
                         float(opacity_scale), float(term_alpha), _ptr(g, C.c_double),
                         _ptr(rgba, C.c_double), _ptr(gv, C.c_double), _ptr(gl, C.c_double),
                         _ptr(gs, C.c_double))
    return rgba.reshape(H, W, 4), gv, gl, float(gs[0])
