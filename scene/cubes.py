"""Seeded synthetic spectral cubes shaped like the paper's workloads.

The paper's real cubes (THINGS NGC 2903, 1024x1024x87; ALMA Antennae, 750x750x70
with NaN mosaic corners; SAMI GAMA-511867, 2 x 50x50x37) are not available, so
these generators stand in for them: i.i.d. N(0,1) noise (sigma = 1 is the noise
unit) plus elliptical Gaussian emission sources whose spectral centroid shifts
linearly with x, mimicking a rotating disc (Section 5.2 data description).

Layout: C-contiguous float32 ``[nz][ny][nx]``; x fastest, z = the spectral axis.
All randomness comes from numpy's PCG64 seeded with ``SEED_BASE + config id``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 1707_00442
FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))  # Eq. 6


def _rng(config_id: int, stream: int = 0) -> np.random.Generator:
    ss = np.random.SeedSequence([SEED_BASE + config_id, stream])
    return np.random.Generator(np.random.PCG64(ss))


@dataclass(frozen=True)
class Source:
    x: float
    y: float
    z: float
    peak: float
    sig_major: float
    sig_minor: float
    pa: float          # position angle of the major axis, radians
    sig_z: float       # spectral width, channels
    grad: float        # centroid shift, channels per voxel of x


def add_source(cube: np.ndarray, s: Source, nsig: float = 4.0) -> None:
    """Add one elliptical Gaussian source in place (float64 math, float32 store)."""
    nz, ny, nx = cube.shape
    ext = nsig * s.sig_major
    x0, x1 = max(0, int(math.floor(s.x - ext))), min(nx, int(math.ceil(s.x + ext)) + 1)
    y0, y1 = max(0, int(math.floor(s.y - ext))), min(ny, int(math.ceil(s.y + ext)) + 1)
    zext = nsig * s.sig_z + abs(s.grad) * ext
    z0, z1 = max(0, int(math.floor(s.z - zext))), min(nz, int(math.ceil(s.z + zext)) + 1)
    if x0 >= x1 or y0 >= y1 or z0 >= z1:
        return
    X = np.arange(x0, x1, dtype=np.float64)[None, None, :]
    Y = np.arange(y0, y1, dtype=np.float64)[None, :, None]
    Z = np.arange(z0, z1, dtype=np.float64)[:, None, None]
    c, sn = math.cos(s.pa), math.sin(s.pa)
    u = (X - s.x) * c + (Y - s.y) * sn
    v = -(X - s.x) * sn + (Y - s.y) * c
    zc = s.z + s.grad * (X - s.x)
    val = s.peak * np.exp(-0.5 * ((u / s.sig_major) ** 2 + (v / s.sig_minor) ** 2)
                          - 0.5 * ((Z - zc) / s.sig_z) ** 2)
    cube[z0:z1, y0:y1, x0:x1] += val.astype(np.float32)


def draw_sources(rng: np.random.Generator, dims, n: int, *, peak=(5.0, 5.0),
                 sig_major=(4.0, 8.0), fwhm_loguniform=None, sig_z=3.0,
                 margin: float = 0.0) -> list[Source]:
    nx, ny, nz = dims
    out = []
    for _ in range(n):
        if fwhm_loguniform is not None:
            lo, hi = fwhm_loguniform
            smaj = math.exp(rng.uniform(math.log(lo), math.log(hi))) / FWHM_PER_SIGMA
        else:
            smaj = rng.uniform(*sig_major)
        smin = smaj * rng.uniform(0.4, 1.0)
        def pos(n):
            lo, hi = margin * n, max(margin * n, (1 - margin) * n - 1)
            return rng.uniform(lo, hi)
        out.append(Source(
            x=pos(nx), y=pos(ny), z=pos(nz),
            peak=rng.uniform(*peak), sig_major=smaj, sig_minor=smin,
            pa=rng.uniform(0.0, math.pi), sig_z=sig_z, grad=rng.uniform(-0.5, 0.5)))
    return out


def _noise(rng: np.random.Generator, dims) -> np.ndarray:
    nx, ny, nz = dims
    return rng.standard_normal((nz, ny, nx), dtype=np.float32)


def tiny_cube(config_id: int = 1, dims=(64, 64, 64), n_sources: int = 3) -> np.ndarray:
    """64^3 noise + 3 sources, peak 5 sigma, spatial sigma U[4,8], spectral sigma 3."""
    rng = _rng(config_id)
    cube = _noise(rng, dims)
    for s in draw_sources(rng, dims, n_sources, margin=0.2):
        add_source(cube, s)
    return cube


def survey_cube(config_id: int = 2, dims=(512, 512, 1024), n_sources: int = 200) -> np.ndarray:
    """Survey-sized cube: noise + sources with FWHM log-uniform in [6,40] vox, peak U[2,10]."""
    rng = _rng(config_id)
    cube = _noise(rng, dims)
    for s in draw_sources(rng, dims, n_sources, peak=(2.0, 10.0), fwhm_loguniform=(6.0, 40.0)):
        add_source(cube, s)
    return cube


def ratio_cube(first: np.ndarray, config_id: int = 2, factor: float = 0.3,
               noise: bool = True) -> np.ndarray:
    """Second co-registered line: ``factor * first`` (+ fresh N(0,1) noise when ``noise``)."""
    out = (first * np.float32(factor)).astype(np.float32)
    if noise:
        out += _noise(_rng(config_id, stream=1), first.shape[::-1])
    return out


def diff_cube(config_id: int = 5, dims=(256, 256, 256), n_sources: int = 10) -> np.ndarray:
    """Differentiation workload: the tiny-cube model scaled to ``dims``."""
    rng = _rng(config_id)
    cube = _noise(rng, dims)
    scale = min(dims[0], dims[1]) / 64.0
    for s in draw_sources(rng, dims, n_sources, sig_major=(4.0 * scale, 8.0 * scale),
                          sig_z=3.0 * dims[2] / 64.0, margin=0.1):
        add_source(cube, s)
    return cube


def batch_dims(n: int = 2000, config_id: int = 4, lo: int = 32, hi: int = 256) -> np.ndarray:
    """Sub-cube dims: each axis floor(exp U(ln lo, ln hi)); returns int array [n, 3] = (nx, ny, nz)."""
    rng = _rng(config_id, stream=7)
    d = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=(n, 3)))).astype(np.int64)
    return np.clip(d, lo, hi)


def batch_subcube(i: int, dims, config_id: int = 4) -> np.ndarray:
    """Sub-cube ``i`` of the batch: noise plus one source of the tiny-cube model, scaled."""
    rng = _rng(config_id, stream=1000 + int(i))
    cube = _noise(rng, dims)
    scale = min(dims[0], dims[1]) / 64.0
    for s in draw_sources(rng, dims, 1, sig_major=(4.0 * scale, 8.0 * scale),
                          sig_z=max(1.0, 3.0 * dims[2] / 64.0), margin=0.25):
        add_source(cube, s)
    return cube


def paper_uniform_cube(n: int, config_id: int = 9) -> np.ndarray:
    """The paper's benchmark cubes: every voxel an independent U[0,1] float32 (Appendix B)."""
    return _rng(config_id, stream=n).random((n, n, n), dtype=np.float32)


# The paper's three real cubes (Section 5.2), stood in for by shape and by the intensity
# range its histograms report, in units of each cube's noise sigma: NGC 2903 1024x1024x87
# (minimum about -7 sigma, maximum about 15 sigma); the Antennae mosaic 750x750x70 (maximum
# about 68 sigma; NaN outside a tilted polygon, the mosaic's footprint); GAMA-511867 two
# 50x50x37 sub-cubes, H-alpha (maximum about 8 sigma) and [NII] (about 7.6 sigma).
STANDIN_DIMS = {"ngc2903": (1024, 1024, 87), "antennae": (750, 750, 70), "gama511867": (50, 50, 37)}


def paper_standin(kind: str, config_id: int = 10) -> np.ndarray | tuple:
    """A stand-in for one of the paper's cubes: N(0,1) noise plus rotating-disc sources whose
    peaks reach the reported maximum.  ``gama511867`` returns the (H-alpha, [NII]) pair, the
    second line 0.4 times the first plus its own noise (a line ratio near 0.4)."""
    dims = STANDIN_DIMS[kind]
    rng = _rng(config_id, stream={"ngc2903": 1, "antennae": 2, "gama511867": 3}[kind])
    cube = _noise(rng, dims)
    nx, ny, nz = dims
    if kind == "ngc2903":
        srcs = draw_sources(rng, dims, 1, peak=(15.0, 15.0), sig_major=(nx / 8, nx / 8), sig_z=nz / 8, margin=0.4)
        srcs += draw_sources(rng, dims, 40, peak=(2.0, 8.0), fwhm_loguniform=(6.0, 40.0), sig_z=3.0)
    elif kind == "antennae":
        srcs = draw_sources(rng, dims, 2, peak=(30.0, 40.0), sig_major=(nx / 20, nx / 12), sig_z=nz / 10, margin=0.3)
        srcs += draw_sources(rng, dims, 30, peak=(2.0, 10.0), fwhm_loguniform=(6.0, 30.0), sig_z=3.0, margin=0.2)
    else:
        srcs = draw_sources(rng, dims, 1, peak=(8.0, 8.0), sig_major=(nx / 6, nx / 6), sig_z=nz / 8, margin=0.4)
    for s in srcs:
        add_source(cube, s)
    if kind == "antennae":
        # the mosaic's footprint: a square tilted by 30 degrees covering the central part
        y, x = np.mgrid[0:ny, 0:nx]
        c, s_ = math.cos(math.radians(30.0)), math.sin(math.radians(30.0))
        u = (x - nx / 2) * c + (y - ny / 2) * s_
        v = -(x - nx / 2) * s_ + (y - ny / 2) * c
        outside = (np.abs(u) > 0.36 * nx) | (np.abs(v) > 0.36 * ny)
        cube[:, outside] = np.nan
    if kind == "gama511867":
        second = (cube * np.float32(0.4)).astype(np.float32) + _noise(_rng(config_id, stream=4), dims)
        return cube, second
    return cube
