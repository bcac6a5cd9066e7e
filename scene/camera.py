"""Camera frames (inputs, float32) for parallel and perspective projection.

A camera is the frame the caller hands to both the CUDA library and the oracle:
eye position, unit right/up/forward vectors in voxel-index space, the tangent of
half the vertical field of view (perspective) or the half height of the view
window in voxels (parallel), and the image size.  How a pixel turns into a ray
is NOT defined here; that is the method's arithmetic (Appendix A projections).

Index space: voxel (i, j, k) of a ``[nz][ny][nx]`` cube sits at the point
(x, y, z) = (i, j, k); the cube's box is [-0.5, n - 0.5] on each axis.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _f32(v):
    return np.asarray(v, dtype=np.float32).reshape(3)


@dataclass
class Camera:
    eye: np.ndarray
    right: np.ndarray
    up: np.ndarray
    fwd: np.ndarray
    tan_half_fovy: float
    ortho_half_h: float
    ortho: bool
    width: int
    height: int
    meta: dict = field(default_factory=dict)

    def vec14(self) -> np.ndarray:
        """eye, right, up, fwd, tan_half_fovy, ortho_half_h as 14 float32 values."""
        return np.concatenate([_f32(self.eye), _f32(self.right), _f32(self.up), _f32(self.fwd),
                               np.array([self.tan_half_fovy, self.ortho_half_h], np.float32)])


def _frame(fwd):
    fwd = np.asarray(fwd, np.float64)
    fwd = fwd / np.linalg.norm(fwd)
    hint = np.array([0.0, 1.0, 0.0])
    if abs(np.dot(hint, fwd)) > 0.999:
        hint = np.array([0.0, 0.0, 1.0])
    right = np.cross(hint, fwd)
    right /= np.linalg.norm(right)
    up = np.cross(fwd, right)
    return right, up, fwd


def ortho_axis_camera(dims, width: int, height: int, axis: str = "z") -> Camera:
    """Parallel projection looking down +axis, window exactly covering the cube's face.

    Looking down +z: image column px covers x in [-0.5, nx-0.5], row 0 at y = ny - 0.5.
    With width = 2 nx the pixel centres land at x = px/2 - 1/4 (no rounding ties).
    """
    nx, ny, nz = dims
    if axis == "z":
        right, up, fwd = (1, 0, 0), (0, 1, 0), (0, 0, 1)
        cx, cy, half_w, half_h = (nx - 1) / 2, (ny - 1) / 2, nx / 2, ny / 2
        eye = (cx, cy, -8.0)
    elif axis == "x":
        right, up, fwd = (0, 0, 1), (0, 1, 0), (1, 0, 0)
        half_w, half_h = nz / 2, ny / 2
        eye = (-8.0, (ny - 1) / 2, (nz - 1) / 2)
    elif axis == "y":
        right, up, fwd = (1, 0, 0), (0, 0, 1), (0, 1, 0)
        half_w, half_h = nx / 2, nz / 2
        eye = ((nx - 1) / 2, -8.0, (nz - 1) / 2)
    else:
        raise ValueError(axis)
    if abs(half_w / half_h - width / height) > 1e-12:
        raise ValueError("aspect of image and cube face differ")
    return Camera(_f32(eye), _f32(right), _f32(up), _f32(fwd), 0.0, float(half_h), True,
                  int(width), int(height), {"kind": "ortho-axis", "axis": axis})


def orbit_camera(dims, yaw_deg: float, pitch_deg: float, width: int, height: int,
                 fov_deg: float = 45.0, ortho: bool = False, dist_scale: float = 1.0) -> Camera:
    """Camera on a sphere around the cube centre, looking at the centre.

    yaw rotates about the y (dec) axis, pitch about x; yaw = pitch = 0 looks down +z
    (the spatial, face-on view).  Distance = R / sin(fov/2), R = half box diagonal,
    so the whole cube fits the view.
    """
    nx, ny, nz = dims
    c = np.array([(nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2])
    R = 0.5 * math.sqrt(nx * nx + ny * ny + nz * nz)
    yaw, pitch = math.radians(yaw_deg), math.radians(pitch_deg)
    fwd = np.array([math.sin(yaw) * math.cos(pitch), math.sin(pitch), math.cos(yaw) * math.cos(pitch)])
    right, up, fwd = _frame(fwd)
    half = math.radians(fov_deg) / 2
    dist = dist_scale * R / math.sin(half)
    eye = c - dist * fwd
    return Camera(_f32(eye), _f32(right), _f32(up), _f32(fwd), float(np.float32(math.tan(half))),
                  float(np.float32(R)), bool(ortho), int(width), int(height),
                  {"kind": "orbit", "yaw": yaw_deg, "pitch": pitch_deg, "fov": fov_deg})
