"""Python binding of libshw: torch tensors in, torch tensors out.

PyTorch supplies device memory and the current CUDA stream; each function here
only checks tensor properties, marshals pointers and sizes into the C ABI
(include/shw.h), and raises ShwError on a non-OK status.  Every step of the
computation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import INTERP, MODES, STORAGE, ShwError, check, lib

__all__ = ["BatchPlan", "BrickVolume", "ShwError", "binomial_taps", "bricked_bytes", "ckpt_bytes", "debug_flags",
           "launch_count", "linear_sampling_taps", "pack_bricks", "render", "render_backward", "smooth",
           "smooth_weights", "smooth_zip", "sync_status"]


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _need_cuda(t: torch.Tensor, name: str, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")


@dataclass
class BrickVolume:
    """A cube packed by ``pack_bricks``: raw 16-bit values (bricks, or a linear 16-bit cube)
    plus the cube's dims."""
    data: torch.Tensor   # int16, shw_bricked_bytes/2 elements
    nx: int
    ny: int
    nz: int
    storage: str          # a key of STORAGE other than "f32" and "pair"

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def volume_struct(vol) -> _lib.Volume:
    if isinstance(vol, BrickVolume):
        _need_cuda(vol.data, "bricks", torch.int16)
        return _lib.Volume(vol.data.data_ptr(), vol.nx, vol.ny, vol.nz, STORAGE[vol.storage])
    _need_cuda(vol, "cube", torch.float32)
    if vol.dim() == 4 and vol.shape[3] == 2:  # the line ratios' interleaved pair storage
        nz, ny, nx, _ = vol.shape
        return _lib.Volume(vol.data_ptr(), nx, ny, nz, STORAGE["pair"])
    if vol.dim() != 3:
        raise ValueError("cube must be [nz, ny, nx] (or [nz, ny, nx, 2] for the pair storage)")
    nz, ny, nx = vol.shape
    return _lib.Volume(vol.data_ptr(), nx, ny, nz, STORAGE["f32"])


def camera_struct(cam) -> _lib.Camera:
    """Any object with eye/right/up/fwd (3 floats), tan_half_fovy, ortho_half_h, ortho, width, height."""
    c = _lib.Camera()
    for name in ("eye", "right", "up", "fwd"):
        v = [float(x) for x in getattr(cam, name)]
        getattr(c, name)[:] = v
    c.tan_half_fovy = float(cam.tan_half_fovy)
    c.ortho_half_h = float(cam.ortho_half_h)
    c.ortho = int(bool(cam.ortho))
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


def params_struct(mode, lut, *, interp="trilinear", step=0.5, lo=-3.0, hi=8.0, opacity_scale=1.0,
                  term_alpha=0.99, ratio_floor=0.0, ckpt_interval=64, filter=None, min_threshold=0.0,
                  max_threshold=0.0, alpha_threshold=False, smooth=None, smooth_arm=0,
                  smooth_taps=None) -> _lib.RenderParams:
    """``smooth``: None, "box" (``smooth_arm`` neighbours each side along the ray) or "taps"
    with ``smooth_taps`` = (c0, offsets, weights), e.g. from linear_sampling_taps()."""
    _need_cuda(lut, "lut", torch.float32)
    if lut.numel() != 4 * _lib.LUT_SIZE:
        raise ValueError("lut must hold 256 RGBA entries")
    p = _lib.RenderParams(MODES[mode], INTERP[interp], float(step), float(lo), float(hi), lut.data_ptr(),
                          float(opacity_scale), float(term_alpha), float(ratio_floor), int(ckpt_interval),
                          _lib.FILTERS[filter], float(min_threshold), float(max_threshold),
                          int(bool(alpha_threshold)))
    p.smooth = _lib.SMOOTH[smooth]
    if p.smooth == 1:
        p.smooth_arm = int(smooth_arm)
    elif p.smooth == 2:
        c0, offs, wts = smooth_taps
        offs, wts = [float(x) for x in offs], [float(x) for x in wts]
        if len(offs) != len(wts) or len(offs) > _lib.MAX_SMOOTH_TAPS:
            raise ValueError(f"smooth_taps: at most {_lib.MAX_SMOOTH_TAPS} offsets, one weight each")
        p.smooth_ntaps = len(offs)
        p.smooth_c0 = float(c0)
        for j, (o, w) in enumerate(zip(offs, wts)):
            p.smooth_offset[j] = o
            p.smooth_weight[j] = w
    return p


def _taps_out(call, what):
    c0, nf = C.c_double(), C.c_int32()
    offs, wts = (C.c_double * 64)(), (C.c_double * 64)()
    check(call(C.byref(c0), offs, wts, 64, C.byref(nf)), what)
    n = nf.value
    return c0.value, list(offs[:n]), list(wts[:n])


def linear_sampling_taps(w):
    """Fold a symmetric 1-D kernel w[-r..r] into the fetches of SHW_SMOOTH_TAPS by linear
    sampling (Section 4.2, Algorithm 9), computed by the library (shw_linear_sampling_taps).
    Returns (c0, offsets, weights)."""
    wl = [float(x) for x in w]
    if len(wl) % 2 != 1:
        raise ValueError("the kernel must have odd length 2r+1")
    arr = (C.c_double * len(wl))(*wl)
    return _taps_out(lambda *o: lib().shw_linear_sampling_taps(arr, (len(wl) - 1) // 2, *o),
                     "shw_linear_sampling_taps")


def binomial_taps(ntaps: int, drop: int = 0):
    """The N-tap binomial filter of Section 4.2 folded for SHW_SMOOTH_TAPS, computed by the
    library (shw_binomial_taps): b_{N-1+2 drop} without its `drop` outer taps on each side,
    renormalised.  ntaps = 5, 9, 13 with drop = 0 are b_4, b_8, b_12; ntaps = 9, drop = 2 is
    the kernel whose folded constants Algorithm 9 prints."""
    return _taps_out(lambda *o: lib().shw_binomial_taps(int(ntaps), int(drop), *o), "shw_binomial_taps")


class debug_flags:
    """Context manager setting the library's test and diagnosis switches (shw_set_debug_flags)
    by name, e.g. ``with debug_flags("no_axis_sweep"): ...``; the previous set is restored."""

    def __init__(self, *names):
        self.mask = 0
        for n in names:
            self.mask |= _lib.DEBUG[n]

    def __enter__(self):
        self.prev = int(lib().shw_set_debug_flags(self.mask))
        return self

    def __exit__(self, *exc):
        lib().shw_set_debug_flags(self.prev)
        return False


def smooth(cube: torch.Tensor, sigma: float, radius: int, out: torch.Tensor | None = None) -> torch.Tensor:
    """Separable 3-D Gaussian smoothing (Eqs. 5-6), clamp-to-edge; see shw_smooth."""
    _need_cuda(cube, "cube", torch.float32)
    out = torch.empty_like(cube) if out is None else out
    _need_cuda(out, "out", torch.float32)
    nz, ny, nx = cube.shape
    check(lib().shw_smooth(cube.data_ptr(), out.data_ptr(), nx, ny, nz, float(sigma), int(radius), _stream()),
          "shw_smooth")
    return out


def smooth_zip(cube: torch.Tensor, first: torch.Tensor, sigma: float, radius: int,
               out: torch.Tensor | None = None) -> torch.Tensor:
    """Smooth ``cube`` as smooth() does and interleave it after ``first``: the [nz, ny, nx, 2]
    pair storage of the line ratios, (first, smoothed) per voxel (shw_smooth_zip)."""
    _need_cuda(cube, "cube", torch.float32)
    _need_cuda(first, "first", torch.float32)
    if cube.dim() != 3 or tuple(first.shape) != tuple(cube.shape):
        raise ValueError("cube and first must be [nz, ny, nx] of the same shape")
    nz, ny, nx = cube.shape
    out = torch.empty((nz, ny, nx, 2), dtype=torch.float32, device=cube.device) if out is None else out
    _need_cuda(out, "out", torch.float32)
    if tuple(out.shape) != (nz, ny, nx, 2):
        raise ValueError("out must be [nz, ny, nx, 2]")
    check(lib().shw_smooth_zip(cube.data_ptr(), first.data_ptr(), out.data_ptr(), nx, ny, nz, float(sigma),
                               int(radius), _stream()), "shw_smooth_zip")
    return out


def smooth_weights(cube: torch.Tensor, w, out: torch.Tensor | None = None) -> torch.Tensor:
    """Separable smoothing with explicit 1-D weights w[2r+1] (e.g. binomial b_n)."""
    _need_cuda(cube, "cube", torch.float32)
    out = torch.empty_like(cube) if out is None else out
    _need_cuda(out, "out", torch.float32)
    wl = [float(x) for x in w]
    if len(wl) % 2 != 1:
        raise ValueError("weights must have odd length 2r+1")
    arr = (C.c_float * len(wl))(*wl)
    nz, ny, nx = cube.shape
    check(lib().shw_smooth_weights(cube.data_ptr(), out.data_ptr(), nx, ny, nz, arr, (len(wl) - 1) // 2,
                                   _stream()), "shw_smooth_weights")
    return out


def bricked_bytes(dims, storage="bf16") -> int:
    nx, ny, nz = dims
    return int(lib().shw_bricked_bytes(nx, ny, nz, STORAGE[storage]))


def pack_bricks(cube: torch.Tensor, storage: str = "bf16") -> BrickVolume:
    """Round a float32 cube to a 16-bit storage (shw_pack_bricks): "bf16" / "f16" are 32^3
    bricks with a 1-voxel apron, "bf16_linear" / "f16_linear" the linear [nz, ny, nx] cube the
    staged marcher copies boxes from.  A [nz, ny, nx, 2] pair buffer (the line ratios'
    storage) packs into the pair form of the same storage, both cubes' 16-bit values in one
    32-bit element ("bf16_pair", "bf16_linear_pair", ...)."""
    _need_cuda(cube, "cube", torch.float32)
    if cube.dim() == 4 and cube.shape[3] == 2:
        nz, ny, nx, _ = cube.shape
        storage = storage if storage.endswith("_pair") else storage + "_pair"
    elif cube.dim() == 3 and not storage.endswith("_pair"):
        nz, ny, nx = cube.shape
    else:
        raise ValueError("pair bricks pack a [nz, ny, nx, 2] pair buffer; a cube must be [nz, ny, nx]")
    nbytes = bricked_bytes((nx, ny, nz), storage)
    data = torch.empty(nbytes // 2, dtype=torch.int16, device=cube.device)
    check(lib().shw_pack_bricks(cube.data_ptr(), nx, ny, nz, STORAGE[storage], data.data_ptr(), nbytes,
                                _stream()), "shw_pack_bricks")
    return BrickVolume(data, nx, ny, nz, storage)


def ckpt_bytes(vol, cam, *, step=0.5, ckpt_interval=64) -> int:
    v, c = volume_struct(vol), camera_struct(cam)
    p = _lib.RenderParams(MODES["composite"], 1, float(step), 0.0, 1.0, None, 1.0, 0.99, 0.0, int(ckpt_interval))
    return int(lib().shw_ckpt_bytes(C.byref(v), C.byref(c), C.byref(p)))


def render(vol, cam, mode: str, *, lut: torch.Tensor, interp="trilinear", step=0.5, lo=-3.0, hi=8.0,
           opacity_scale=1.0, term_alpha=0.99, ratio_floor=0.0, vol2=None, scalar=True, index=True,
           nsamples=True, ckpt=False, ckpt_interval=64, out=None, filter=None, min_threshold=0.0,
           max_threshold=0.0, alpha_threshold=False, smooth=None, smooth_arm=0, smooth_taps=None) -> dict:
    """Render one image (shw_render).  Returns a dict of CUDA tensors:
    rgba [H, W, 4] and optionally scalar [H, W], index [H, W], nsamples [H, W], ckpt (bytes).
    ``out``: optional dict of preallocated tensors with the same keys."""
    v = volume_struct(vol)
    v2 = volume_struct(vol2) if vol2 is not None else None
    c = camera_struct(cam)
    p = params_struct(mode, lut, interp=interp, step=step, lo=lo, hi=hi, opacity_scale=opacity_scale,
                      term_alpha=term_alpha, ratio_floor=ratio_floor, ckpt_interval=ckpt_interval, filter=filter,
                      min_threshold=min_threshold, max_threshold=max_threshold, alpha_threshold=alpha_threshold,
                      smooth=smooth, smooth_arm=smooth_arm, smooth_taps=smooth_taps)
    dev = lut.device
    H, W = c.height, c.width
    out = dict(out or {})

    def get(key, shape, dtype, want):
        if not want:
            return None
        t = out.get(key)
        if t is None:
            t = torch.empty(shape, dtype=dtype, device=dev)
            out[key] = t
        _need_cuda(t, key, dtype)
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{key} must have shape {shape}")
        return t

    rgba = get("rgba", (H, W, 4), torch.float32, True)
    sc = get("scalar", (H, W), torch.float32, scalar)
    ix = get("index", (H, W), torch.int32, index)
    ns = get("nsamples", (H, W), torch.int32, nsamples)
    ck = None
    nck = 0
    if ckpt:
        nck = int(lib().shw_ckpt_bytes(C.byref(v), C.byref(c), C.byref(p)))
        ck = get("ckpt", (nck,), torch.uint8, True)
    ptr = lambda t: None if t is None else t.data_ptr()
    check(lib().shw_render(C.byref(v), C.byref(v2) if v2 is not None else None, C.byref(c), C.byref(p),
                           ptr(rgba), ptr(sc), ptr(ix), ptr(ns), ptr(ck), nck, _stream()), "shw_render")
    return out


def render_backward(vol, cam, grad_rgba: torch.Tensor, ckpt: torch.Tensor, *, lut: torch.Tensor, interp="trilinear",
                    step=0.5, lo=-3.0, hi=8.0, opacity_scale=1.0, term_alpha=0.99, ckpt_interval=64,
                    grad_vol: torch.Tensor | None = None, grad_lut: torch.Tensor | None = None,
                    grad_scale: torch.Tensor | None = None) -> None:
    """Accumulate (+=) the gradient of a compositing render into grad_vol / grad_lut / grad_scale
    (shw_render_backward).  ``ckpt`` is the buffer returned by ``render(..., ckpt=True)`` with the
    same arguments."""
    v, c = volume_struct(vol), camera_struct(cam)
    p = params_struct("composite", lut, interp=interp, step=step, lo=lo, hi=hi, opacity_scale=opacity_scale,
                      term_alpha=term_alpha, ckpt_interval=ckpt_interval)
    _need_cuda(grad_rgba, "grad_rgba", torch.float32)
    _need_cuda(ckpt, "ckpt", torch.uint8)
    for t, name in ((grad_vol, "grad_vol"), (grad_lut, "grad_lut"), (grad_scale, "grad_scale")):
        if t is not None:
            _need_cuda(t, name, torch.float32)
    ptr = lambda t: None if t is None else t.data_ptr()
    check(lib().shw_render_backward(C.byref(v), C.byref(c), C.byref(p), grad_rgba.data_ptr(), ckpt.data_ptr(),
                                    ckpt.numel(), ptr(grad_vol), ptr(grad_lut), ptr(grad_scale), _stream()),
          "shw_render_backward")


class BatchPlan:
    """A plan rendering many sub-cubes with one CUDA-graph launch (shw_batch_plan_create).

    items: sequence of (vol, cam, mode) or (vol, cam, mode, out_rgba); vol is a float32 CUDA
    cube or a BrickVolume; mode one of "mip", "avg", "composite", "spectral".  Missing
    outputs are allocated.  The plan keeps references to every tensor it points at.
    pack: None, "bf16" or "f16" -- the plan rounds the float32 items into 16-bit bricks it
    owns; brick: None (the autotuner picks 16 or 32 when every item is packed), 16 or 32."""

    def __init__(self, items, *, lut: torch.Tensor, interp="trilinear", step=0.5, lo=-3.0, hi=8.0,
                 opacity_scale=1.0, term_alpha=0.99, tune=True, retune=False, pack=None, brick=None):
        self._plan = None
        p = params_struct("mip", lut, interp=interp, step=step, lo=lo, hi=hi, opacity_scale=opacity_scale,
                          term_alpha=term_alpha)
        arr = (_lib.BatchItem * len(items))()
        self.outputs, self._keep = [], [lut]
        for i, it in enumerate(items):
            vol, cam, mode = it[0], it[1], it[2]
            out = it[3] if len(it) > 3 and it[3] is not None else torch.empty(
                (int(cam.height), int(cam.width), 4), dtype=torch.float32, device=lut.device)
            _need_cuda(out, "out_rgba", torch.float32)
            arr[i].vol = volume_struct(vol)
            arr[i].cam = camera_struct(cam)
            arr[i].out_rgba = out.data_ptr()
            arr[i].mode = MODES[mode]
            self.outputs.append(out)
            self._keep.append(vol)
        flags = ((0 if tune else _lib.BATCH_NO_TUNE) | (_lib.BATCH_RETUNE if retune else 0) | _lib.BATCH_PACK[pack]
                 | _lib.BATCH_BRICK[brick])
        handle = C.c_void_p()
        check(lib().shw_batch_plan_create(C.byref(handle), arr, len(items), C.byref(p), flags, _stream()),
              "shw_batch_plan_create")
        self._plan = handle
        self._items, self._params = arr, p

    def render_one_by_one(self) -> list:
        """The same images with one launch per item, looped inside the library
        (shw_render_items): the unbatched path the plan is measured against."""
        check(lib().shw_render_items(self._items, len(self._items), C.byref(self._params), _stream()),
              "shw_render_items")
        return self.outputs

    def render(self) -> list:
        check(lib().shw_render_batch(self._plan, _stream()), "shw_render_batch")
        return self.outputs

    @property
    def info(self) -> dict:
        inf = _lib.BatchInfo()
        check(lib().shw_batch_plan_info(self._plan, C.byref(inf)), "shw_batch_plan_info")
        n = inf.n_candidates
        return {"n_items": inf.n_items, "n_work": inf.n_work, "tile": inf.tile, "ctas_per_sm": inf.ctas_per_sm,
                "grid": inf.grid, "tuned": bool(inf.tuned), "brick": inf.brick, "packed_bytes": int(inf.packed_bytes),
                "candidates": [(inf.cand_tile[i], inf.cand_ctas_per_sm[i], inf.cand_brick[i], float(inf.tune_ms[i]))
                               for i in range(n)]}

    def close(self):
        if self._plan is not None:
            lib().shw_batch_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sync_status() -> None:
    check(lib().shw_sync_status(_stream()), "shw_sync_status")


def launch_count() -> int:
    return int(lib().shw_launch_count())
