"""The line ratios on the interleaved pair storage (both cubes in one [nz, ny, nx, 2] buffer,
written by shw_smooth_zip): the same images as the two-cube render bit for bit, and the
oracle's within the FP32 tolerance; shw_smooth_zip interleaves exactly shw_smooth's values."""
import numpy as np
import pytest
import torch

import oracle
import scene
from parity import compare, gpu_render, shw, to_dev

pytestmark = pytest.mark.gpu

RAGGED_DIMS = (61, 53, 47)


@pytest.fixture(scope="module")
def m():
    return shw()


@pytest.fixture(scope="module")
def ragged():
    c = scene.tiny_cube(config_id=11, dims=RAGGED_DIMS, n_sources=4)
    return c, scene.ratio_cube(c, config_id=11)


def _pair(c1, c2):
    return to_dev(np.stack([c1, c2], axis=-1))


@pytest.mark.parametrize("dims", [(64, 64, 64), RAGGED_DIMS, (96, 40, 33)])
@pytest.mark.parametrize("sigma,radius", [(1.0, 3), (2.0, 6), (4.0, 12)])
def test_smooth_zip_interleaves_smooth(m, dims, sigma, radius):
    cube = scene.tiny_cube(config_id=5, dims=dims, n_sources=2)
    first = scene.ratio_cube(cube, config_id=5)
    ct, ft = to_dev(cube), to_dev(first)
    z = m.smooth_zip(ct, ft, sigma, radius)
    s = m.smooth(ct, sigma, radius)
    torch.cuda.synchronize()
    m.sync_status()
    z, s = z.cpu().numpy(), s.cpu().numpy()
    assert np.array_equal(z[..., 0], first)
    assert np.array_equal(z[..., 1], s)


@pytest.mark.parametrize("mode", ["ratio", "ratio_mip"])
@pytest.mark.parametrize("interp", ["trilinear", "nearest"])
@pytest.mark.parametrize("view", ["persp", "ortho_oblique", "axis"])
def test_pair_render_equals_two_cube_render(m, ragged, mode, interp, view):
    c1, c2 = ragged
    if view == "persp":
        cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 100, 75)
    elif view == "axis":
        cam = scene.ortho_axis_camera(RAGGED_DIMS, 2 * RAGGED_DIMS[0], 2 * RAGGED_DIMS[1])
    else:
        cam = scene.orbit_camera(RAGGED_DIMS, -52, 33, 90, 70, ortho=True)
    lut = scene.ratio_lut()
    kw = dict(lo=0.0, hi=1.0, ratio_floor=1.0, interp=interp)
    two = gpu_render(m, to_dev(c1), cam, mode, to_dev(lut), vol2=to_dev(c2), **kw)
    one = gpu_render(m, _pair(c1, c2), cam, mode, to_dev(lut), **kw)
    for k in two:
        assert np.array_equal(two[k], one[k]), k
    o = oracle.render(c1, cam, mode, lut=lut, cube2=c2, eps_pos=1e-6, eps_val=1e-4, **kw)
    scale = float(o["scalar"].max() - o["scalar"].min()) or 1.0
    compare(one, o, mode, scale=scale, max_fragile=0.05, what=f"pair/{mode}/{interp}/{view}")


def test_pair_render_with_filter_and_nan(m, ragged):
    c1, c2 = ragged
    c1 = c1.copy()
    c1.reshape(-1)[np.random.default_rng(2).integers(0, c1.size, 50)] = np.nan
    cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 80, 60)
    lut = to_dev(scene.ratio_lut())
    kw = dict(lo=0.0, hi=1.0, ratio_floor=1.0, filter="clip", min_threshold=0.5, max_threshold=6.0)
    for mode in ("ratio", "ratio_mip"):
        two = gpu_render(m, to_dev(c1), cam, mode, lut, vol2=to_dev(c2), **kw)
        one = gpu_render(m, _pair(c1, c2), cam, mode, lut, **kw)
        for k in two:
            assert np.array_equal(two[k], one[k]), (mode, k)


def test_pair_from_smooth_zip_matches_two_smoothed_cubes(m, ragged):
    """The survey step's form: smooth the first cube, smooth the second into the pair
    storage, render the ratio -- the same image as rendering the two smoothed cubes."""
    c1, c2 = ragged
    s1 = m.smooth(to_dev(c1), 2.0, 6)
    s2 = m.smooth(to_dev(c2), 2.0, 6)
    pr = m.smooth_zip(to_dev(c2), s1, 2.0, 6)
    cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 80, 60)
    lut = to_dev(scene.ratio_lut())
    kw = dict(lo=0.0, hi=1.0, ratio_floor=0.5)
    two = gpu_render(m, s1, cam, "ratio", lut, vol2=s2, **kw)
    one = gpu_render(m, pr, cam, "ratio", lut, **kw)
    for k in two:
        assert np.array_equal(two[k], one[k]), k


def test_pair_storage_rejections(m, ragged):
    c1, c2 = ragged
    pr = _pair(c1, c2)
    cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 32, 24)
    lut = to_dev(scene.linear_lut())
    with pytest.raises(m.ShwError) as e:
        m.render(pr, cam, "mip", lut=lut)
    assert e.value.status == 2
    with pytest.raises(m.ShwError) as e:
        m.render(pr, cam, "ratio", lut=lut, vol2=to_dev(c2))
    assert e.value.status == 1
    with pytest.raises(m.ShwError) as e:
        m.render(pr, cam, "ratio", lut=lut, smooth="box", smooth_arm=1)
    assert e.value.status == 2
    torch.cuda.synchronize()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("mode", ["ratio", "ratio_mip"])
@pytest.mark.parametrize("interp", ["trilinear", "nearest"])
def test_pair_bricks_equal_two_brick_render(m, storage, mode, interp):
    """Pair bricks (both cubes' 16-bit values in one 32-bit element) render the line ratios
    exactly like two separate brick volumes, and like the oracle on the rounded cubes."""
    dims = (70, 45, 66)
    c1 = scene.tiny_cube(config_id=33, dims=dims, n_sources=3)
    c2 = scene.ratio_cube(c1, config_id=33)
    cam = scene.orbit_camera(dims, -25, 30, 80, 64)
    lut = scene.ratio_lut()
    kw = dict(lo=0.0, hi=1.0, ratio_floor=1.0, interp=interp)
    pb = m.pack_bricks(_pair(c1, c2), storage)
    assert pb.storage == storage + "_pair"
    one = gpu_render(m, pb, cam, mode, to_dev(lut), **kw)
    two = gpu_render(m, m.pack_bricks(to_dev(c1), storage), cam, mode, to_dev(lut),
                     vol2=m.pack_bricks(to_dev(c2), storage), **kw)
    for k in two:
        assert np.array_equal(two[k], one[k]), k
    rnd = oracle.round_bf16 if storage == "bf16" else oracle.round_f16
    o = oracle.render(rnd(c1), cam, mode, lut=lut, cube2=rnd(c2), eps_pos=1e-6, eps_val=1e-4, **kw)
    scale = float(o["scalar"].max() - o["scalar"].min()) or 1.0
    compare(one, o, mode, scale=scale, max_fragile=0.05, what=f"{storage}_pair/{mode}/{interp}")
