"""Pins of the oracle's position-coloured transfer functions and the line ratio Method 1:
AVIP_1 (Algorithm 5: compositing coloured by the sample's spectral position), MIP_RGB and
AVIP_RGB (Algorithms 6-7: (r, g, b) = the position (z, y, x) as texture coordinates) and
Method 1 of the line ratio (Algorithms 12-13: the ratio of the two cubes' maxima).
Each restates the definition in numpy on the spectral-axis view with nearest sampling,
where sample k of a ray sits in channel k // 2 of its pixel's voxel column."""
import numpy as np
import pytest

import scene

LO, HI = -3.0, 8.0


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


@pytest.fixture(scope="module")
def tiny():
    return scene.tiny_cube()


CAM = scene.ortho_axis_camera((64, 64, 64), 128, 128)


def _img(m):
    return m[::-1, :].repeat(2, 0).repeat(2, 1)


def _tex(i, n):
    return np.clip((np.asarray(i, np.float64) + 0.5) / n, 0, 1)


def _lut(u):
    lut = scene.linear_lut().astype(np.float64)
    u = 255 * np.clip(u, 0, 1)
    i0 = np.minimum(np.floor(u).astype(int), 254)
    f = (u - i0)[..., None]
    return (1 - f) * lut[i0] + f * lut[i0 + 1]


def test_mip_rgb_colour_is_position_of_last_maximum(O, tiny):
    cube = np.round(tiny * 2).astype(np.float32)  # exact ties: the last maximum wins
    r = O.render(cube, CAM, "mip_rgb", interp="nearest", lut=scene.linear_lut(), lo=LO, hi=HI)
    last = 63 - np.argmax(cube[::-1], axis=0)
    yy, xx = np.meshgrid(np.arange(64), np.arange(64), indexing="ij")
    assert np.array_equal(r["rgba"][..., 0], _img(_tex(last, 64)))
    assert np.array_equal(r["rgba"][..., 1], _img(_tex(yy, 64)))
    assert np.array_equal(r["rgba"][..., 2], _img(_tex(xx, 64)))
    vhat = np.clip((cube.astype(np.float64).max(axis=0) - LO) / (HI - LO), 0, 1)
    assert np.allclose(r["rgba"][..., 3], _img(vhat), rtol=0, atol=1e-15)
    assert np.array_equal(r["index"], _img(last))


@pytest.mark.parametrize("mode", ["composite_spectral", "composite_rgb"])
def test_position_coloured_compositing_constant_cube(O, mode):
    """A constant cube gives every sample the same opacity a, so the colour is
    sum_k a (1 - a)^k colour(z_k, y, x) until alpha passes 0.99."""
    v0, s = 2.0, 0.3
    cube = np.full((16, 8, 8), v0, np.float32)
    cam = scene.ortho_axis_camera((8, 8, 16), 16, 16)
    r = O.render(cube, cam, mode, interp="nearest", lut=scene.linear_lut(), lo=LO, hi=HI, opacity_scale=s)
    a = min(max(s * float(_lut((v0 - LO) / (HI - LO))[3]), 0.0), 1.0)  # the map's alpha (float32 knots)
    ch = np.arange(32) // 2  # sample k -> channel
    T = (1 - a) ** np.arange(32)
    stop = int(np.argmax(1 - (1 - a) ** np.arange(1, 33) > 0.99)) + 1
    w = (a * T)[:stop]
    yy, xx = np.meshgrid(np.arange(8), np.arange(8), indexing="ij")
    if mode == "composite_spectral":
        col = _lut(_tex(ch, 16))[:stop, :3]
        rgb = np.broadcast_to((w[:, None] * col).sum(axis=0), (8, 8, 3))
    else:
        z = (w * _tex(ch, 16)[:stop]).sum()
        rgb = np.stack([np.full((8, 8), z), w.sum() * _tex(yy, 8), w.sum() * _tex(xx, 8)], axis=-1)
    ref = rgb[::-1].repeat(2, 0).repeat(2, 1)
    assert np.allclose(r["rgba"][..., :3], ref, rtol=0, atol=1e-13)
    assert np.allclose(r["rgba"][..., 3], 1 - (1 - a) ** stop, rtol=0, atol=1e-14)
    assert (r["nsamples"] == stop).all()


def test_ratio_method1_is_ratio_of_maxima(O, tiny):
    c2 = scene.ratio_cube(tiny, config_id=1)
    floor = 3.0
    r = O.render(tiny, CAM, "ratio_mip", interp="nearest", lut=scene.ratio_lut(), cube2=c2, lo=0.0, hi=1.0,
                 ratio_floor=floor)
    m1 = tiny.astype(np.float64).max(axis=0)
    m2 = c2.astype(np.float64).max(axis=0)
    ok = m1 > floor
    q = np.where(ok, m2 / np.where(ok, m1, 1.0), 0.0)
    assert np.allclose(r["scalar"], _img(np.where(ok, q, 0.0)), rtol=0, atol=1e-14)  # DATAMIN = lo = 0
    rgba = _lut(np.clip(q, 0, 1))
    rgba[~ok] = 0.0
    assert np.allclose(r["rgba"], np.stack([_img(rgba[..., i]) for i in range(4)], axis=-1), rtol=0, atol=1e-13)
    assert (r["index"] == -1).all() and ok.any() and (~ok).any()
