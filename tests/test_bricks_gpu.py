"""Reduced-precision brick storage: packing is bit-exact, and renders from bricks match the
oracle within 2e-3 of the data range (and within 1e-5 of the oracle run on the rounded cube)."""
import numpy as np
import pytest
import torch

import oracle
import scene
from parity import TOL_F32, TOL_REDUCED, compare, gpu_render, shw, to_dev

pytestmark = pytest.mark.gpu

ROUND = {"bf16": oracle.round_bf16, "f16": oracle.round_f16}


@pytest.fixture(scope="module")
def m():
    return shw()


def expected_bricks(cube, storage):
    """All stored elements, from the layout written in shw.h: brick (bx,by,bz), local (lx,ly,lz)
    holds voxel (32b + l - 1) clamped, rounded to nearest even."""
    nz, ny, nx = cube.shape
    nb = [-(-n // 32) for n in (nx, ny, nz)]
    l = np.arange(34)
    X = np.clip(np.arange(nb[0])[:, None] * 32 + l[None, :] - 1, 0, nx - 1)  # [nbx, 34]
    Y = np.clip(np.arange(nb[1])[:, None] * 32 + l[None, :] - 1, 0, ny - 1)
    Z = np.clip(np.arange(nb[2])[:, None] * 32 + l[None, :] - 1, 0, nz - 1)
    r = ROUND[storage](cube)
    # [bz, by, bx, lz, ly, lx]
    e = r[Z[:, None, None, :, None, None], Y[None, :, None, None, :, None], X[None, None, :, None, None, :]]
    bits = e.view(np.uint32)
    if storage == "bf16":
        return (bits >> 16).astype(np.uint16).reshape(-1)
    return e.astype(np.float16).view(np.uint16).reshape(-1)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("dims", [(64, 64, 64), (45, 70, 33), (1, 1, 1), (32, 32, 33)])
def test_pack_bit_exact(m, storage, dims):
    cube = scene.tiny_cube(config_id=31, dims=dims, n_sources=1) * np.float32(3.0)
    b = m.pack_bricks(to_dev(cube), storage)
    m.sync_status()
    got = b.data.cpu().numpy().view(np.uint16)
    assert got.size * 2 == m.bricked_bytes(dims, storage)
    assert np.array_equal(got, expected_bricks(cube, storage))


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("mode", ["mip", "avg", "composite", "spectral", "ratio"])
@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_brick_render_parity(m, storage, mode, interp):
    dims = (70, 45, 66)  # crosses brick faces, ragged bricks
    cube = scene.tiny_cube(config_id=32, dims=dims, n_sources=3)
    c2 = scene.ratio_cube(cube, config_id=32)
    cam = scene.orbit_camera(dims, 35, 25, 96, 72)
    lut = scene.ratio_lut() if mode == "ratio" else scene.linear_lut()
    kw = dict(lo=0.0, hi=1.0, ratio_floor=1.0) if mode == "ratio" else (
        dict(opacity_scale=0.05) if mode == "composite" else {})
    bv = m.pack_bricks(to_dev(cube), storage)
    bv2 = m.pack_bricks(to_dev(c2), storage)
    g = gpu_render(m, bv, cam, mode, to_dev(lut), interp=interp, vol2=bv2, **kw)
    rc, rc2 = ROUND[storage](cube), ROUND[storage](c2)
    o_r = oracle.render(rc, cam, mode, interp=interp, lut=lut, cube2=rc2, eps_pos=1e-6, eps_val=1e-4, **kw)
    sc = float(cube.max() - cube.min())
    # against the unrounded cube, decisions within the reduced-precision bound count as near-ties
    o = oracle.render(cube, cam, mode, interp=interp, lut=lut, cube2=c2, eps_pos=1e-6,
                      eps_val=0.01 if mode == "ratio" else TOL_REDUCED * sc, **kw)

    def scale(oo):
        if mode == "ratio":
            return float(oo["scalar"].max() - oo["scalar"].min()) or 1.0
        return 1.0 if mode == "composite" else sc

    # same arithmetic as the FP32 path on the rounded values
    compare(g, o_r, mode, scale=scale(o_r), what=f"{storage}/{mode}/{interp} vs rounded")
    if mode == "ratio":
        # each interpolated value carries at most u * M of rounding error (u: unit roundoff of the
        # storage, M: the largest corner magnitude); a ratio c2/c1 with c1 > floor then errs by at
        # most u M (1 + |r|) / floor.  Checked on rays whose threshold decisions are not within
        # the rounding margin.
        u = 2.0 ** -8 if storage == "bf16" else 2.0 ** -11
        M = float(max(np.abs(cube).max(), np.abs(c2).max()))
        ok = (o["fragile"].reshape(-1) & 4) == 0
        gs = g["scalar"].reshape(-1)[ok].astype(np.float64)
        os_ = o["scalar"].reshape(-1)[ok]
        assert (np.abs(gs - os_) <= 1.05 * u * M * (1 + np.abs(os_)) / kw["ratio_floor"] + TOL_F32).all()
        return
    # against the unrounded cube: the reduced-precision bound
    compare(g, o, mode, scale=scale(o), tol=TOL_REDUCED, max_fragile=0.5, what=f"{storage}/{mode}/{interp} vs fp32")


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("mode", ["moment1", "composite_spectral", "mip_rgb", "composite_rgb", "ratio_mip"])
def test_brick_render_parity_other_modes(m, storage, mode):
    """The first moment, the position-coloured modes and the ratio Method 1 on bricks: the
    FP32 arithmetic on the rounded values (against the oracle on the rounded cube)."""
    dims = (70, 45, 66)
    cube = scene.tiny_cube(config_id=33, dims=dims, n_sources=3)
    c2 = scene.ratio_cube(cube, config_id=33)
    cam = scene.orbit_camera(dims, -25, 30, 80, 64)
    lut = scene.ratio_lut() if mode == "ratio_mip" else scene.linear_lut()
    kw = dict(lo=0.0, hi=1.0, ratio_floor=1.0) if mode == "ratio_mip" else (
        dict(opacity_scale=0.05) if mode.startswith("composite") else {})
    g = gpu_render(m, m.pack_bricks(to_dev(cube), storage), cam, mode, to_dev(lut),
                   vol2=m.pack_bricks(to_dev(c2), storage), **kw)
    rc, rc2 = ROUND[storage](cube), ROUND[storage](c2)
    o = oracle.render(rc, cam, mode, lut=lut, cube2=rc2, eps_pos=1e-6, eps_val=1e-4, **kw)
    if mode == "ratio_mip":
        scale = float(o["scalar"].max() - o["scalar"].min()) or 1.0
    elif mode == "moment1":
        scale = float(dims[2])
    else:
        scale = 1.0 if mode.startswith("composite") else float(cube.max() - cube.min())
    compare(g, o, mode, scale=scale, max_fragile=0.05, what=f"{storage}/{mode} vs rounded")
