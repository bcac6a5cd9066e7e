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

__all__ = ["BrickVolume", "ShwError", "bricked_bytes", "ckpt_bytes", "launch_count", "pack_bricks", "render",
           "smooth", "smooth_weights", "sync_status"]


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
    """A cube packed by ``pack_bricks``: raw 16-bit bricks plus the cube's dims."""
    data: torch.Tensor   # int16, shw_bricked_bytes/2 elements
    nx: int
    ny: int
    nz: int
    storage: str          # "bf16" | "f16"

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def volume_struct(vol) -> _lib.Volume:
    if isinstance(vol, BrickVolume):
        _need_cuda(vol.data, "bricks", torch.int16)
        return _lib.Volume(vol.data.data_ptr(), vol.nx, vol.ny, vol.nz, STORAGE[vol.storage])
    _need_cuda(vol, "cube", torch.float32)
    if vol.dim() != 3:
        raise ValueError("cube must be [nz, ny, nx]")
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
                  term_alpha=0.99, ratio_floor=0.0, ckpt_interval=64) -> _lib.RenderParams:
    _need_cuda(lut, "lut", torch.float32)
    if lut.numel() != 4 * _lib.LUT_SIZE:
        raise ValueError("lut must hold 256 RGBA entries")
    return _lib.RenderParams(MODES[mode], INTERP[interp], float(step), float(lo), float(hi), lut.data_ptr(),
                             float(opacity_scale), float(term_alpha), float(ratio_floor), int(ckpt_interval))


def smooth(cube: torch.Tensor, sigma: float, radius: int, out: torch.Tensor | None = None) -> torch.Tensor:
    """Separable 3-D Gaussian smoothing (Eqs. 5-6), clamp-to-edge; see shw_smooth."""
    _need_cuda(cube, "cube", torch.float32)
    out = torch.empty_like(cube) if out is None else out
    _need_cuda(out, "out", torch.float32)
    nz, ny, nx = cube.shape
    check(lib().shw_smooth(cube.data_ptr(), out.data_ptr(), nx, ny, nz, float(sigma), int(radius), _stream()),
          "shw_smooth")
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
    """Round a float32 cube to bf16/f16 32^3 bricks with a 1-voxel apron (shw_pack_bricks)."""
    _need_cuda(cube, "cube", torch.float32)
    nz, ny, nx = cube.shape
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
           nsamples=True, ckpt=False, ckpt_interval=64, out=None) -> dict:
    """Render one image (shw_render).  Returns a dict of CUDA tensors:
    rgba [H, W, 4] and optionally scalar [H, W], index [H, W], nsamples [H, W], ckpt (bytes).
    ``out``: optional dict of preallocated tensors with the same keys."""
    v = volume_struct(vol)
    v2 = volume_struct(vol2) if vol2 is not None else None
    c = camera_struct(cam)
    p = params_struct(mode, lut, interp=interp, step=step, lo=lo, hi=hi, opacity_scale=opacity_scale,
                      term_alpha=term_alpha, ratio_floor=ratio_floor, ckpt_interval=ckpt_interval)
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


def sync_status() -> None:
    check(lib().shw_sync_status(_stream()), "shw_sync_status")


def launch_count() -> int:
    return int(lib().shw_launch_count())
