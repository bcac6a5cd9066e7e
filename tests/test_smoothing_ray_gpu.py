"""GPU parity of in-ray smoothing (Section 4.1-4.2: the box along the ray of Algorithm 8 and
the per-axis taps of Algorithm 9, chained x, y, z) against the FP64 oracle, through the
C ABI, for every transfer function, both interpolations, the linear FP32 cube and the
16-bit bricks."""
import numpy as np
import pytest

import oracle
import scene
from parity import TOL_F32, TOL_REDUCED, compare, gpu_render, shw, to_dev

pytestmark = pytest.mark.gpu

MODES = ["mip", "avg", "composite", "spectral", "ratio", "moment1", "composite_spectral", "mip_rgb",
         "composite_rgb", "ratio_mip"]
RAGGED_DIMS = (61, 53, 47)


def _taps(name):
    from paper_1707_00442_gb300 import binomial_taps
    return {"taps9": binomial_taps(9, drop=2), "taps5": binomial_taps(5), "taps13": binomial_taps(13)}[name]


def _smooth(name):
    if name.startswith("box"):
        return dict(smooth="box", smooth_arm=int(name[3:]))
    return dict(smooth="taps", smooth_taps=_taps(name))


@pytest.fixture(scope="module")
def m():
    return shw()


@pytest.fixture(scope="module")
def ragged():
    c = scene.tiny_cube(config_id=7, dims=RAGGED_DIMS, n_sources=3)
    return c, scene.ratio_cube(c, config_id=7)


def _kw(mode):
    if mode.startswith("ratio"):
        return dict(lo=0.0, hi=1.0, ratio_floor=1.0)
    if mode.startswith("composite"):
        return dict(opacity_scale=0.05)
    return {}


def _scale(cube, mode, o):
    if mode.startswith("ratio"):
        s = o["scalar"]
        return float(s.max() - s.min()) or 1.0
    if mode.startswith("composite"):
        return 1.0
    if mode == "moment1":
        return float(cube.shape[0])
    return float(np.nanmax(cube) - np.nanmin(cube))


def _both(m, cube, c2, cam, mode, interp, sm, **extra):
    lut = scene.ratio_lut() if mode.startswith("ratio") else scene.linear_lut()
    kw = dict(_kw(mode), **extra)
    g = gpu_render(m, to_dev(cube), cam, mode, to_dev(lut), interp=interp, vol2=to_dev(c2), **kw, **sm)
    o = oracle.render(cube, cam, mode, interp=interp, lut=lut, cube2=c2, eps_pos=1e-6, eps_val=1e-4, **kw, **sm)
    return g, o


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("kind", ["box2", "taps9"])
@pytest.mark.parametrize("interp", ["trilinear", "nearest"])
def test_smoothing_parity_perspective(m, ragged, mode, kind, interp):
    cube, c2 = ragged
    cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 100, 75)
    g, o = _both(m, cube, c2, cam, mode, interp, _smooth(kind))
    compare(g, o, mode, scale=_scale(cube, mode, o), max_fragile=0.05, what=f"{mode}/{kind}/{interp}")


@pytest.mark.parametrize("kind", ["box1", "box4", "box16", "taps5", "taps13"])
@pytest.mark.parametrize("mode", ["mip", "avg", "composite"])
def test_smoothing_kernel_sizes(m, ragged, kind, mode):
    cube, c2 = ragged
    cam = scene.orbit_camera(RAGGED_DIMS, -50, -15, 64, 48, ortho=True)
    g, o = _both(m, cube, c2, cam, mode, "trilinear", _smooth(kind))
    compare(g, o, mode, scale=_scale(cube, mode, o), max_fragile=0.05, what=f"{mode}/{kind}")


@pytest.mark.parametrize("mode", ["mip", "avg", "spectral"])
def test_smoothing_spectral_axis_view(m, ragged, mode):
    """The spectral-axis view, which without smoothing takes the plane sweep: with smoothing
    it takes the general marcher (the smoothed sums are FP32 arithmetic, so not bit-exact)."""
    cube, c2 = ragged
    nx, ny, nz = RAGGED_DIMS
    cam = scene.ortho_axis_camera(RAGGED_DIMS, 2 * nx, 2 * ny)
    for sm in (_smooth("box3"), _smooth("taps9")):
        g, o = _both(m, cube, c2, cam, mode, "nearest", sm, step=1.0)
        compare(g, o, mode, scale=_scale(cube, mode, o), max_fragile=0.05, what=f"{mode}/{sm['smooth']}")


def test_smoothing_filters_after(m, ragged):
    """Smoothing, then the clip filter (Algorithm 1's order)."""
    cube, c2 = ragged
    cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 80, 60)
    g, o = _both(m, cube, c2, cam, "mip", "trilinear", _smooth("box2"), filter="clip", min_threshold=0.2,
                 max_threshold=2.0)
    compare(g, o, "mip", scale=_scale(cube, "mip", o), max_fragile=0.05, what="box/clip")


def test_smoothing_with_nan_voxels(m, ragged):
    """A NaN voxel inside a tap's reach makes the smoothed sample NaN, then DATAMIN."""
    cube, c2 = ragged
    cube = cube.copy()
    rng = np.random.default_rng(5)
    idx = rng.integers(0, cube.size, 60)
    cube.reshape(-1)[idx] = np.nan
    cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 80, 60)
    for mode in ("mip", "avg", "composite"):
        g, o = _both(m, cube, c2, cam, mode, "trilinear", _smooth("taps9"))
        compare(g, o, mode, scale=1.0 if mode == "composite" else float(np.nanmax(cube) - np.nanmin(cube)),
                max_fragile=0.05, what=f"nan/{mode}")


def test_smoothing_identity_cases(m, ragged):
    """arm 0 and a unit-centre tap table are the unsmoothed render, bit for bit."""
    cube, c2 = ragged
    cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 80, 60)
    lut = to_dev(scene.linear_lut())
    for mode in ("mip", "composite"):
        kw = _kw(mode)
        raw = gpu_render(m, to_dev(cube), cam, mode, lut, **kw)
        for sm in (dict(smooth="box", smooth_arm=0), dict(smooth="taps", smooth_taps=(1.0, [1.5], [0.0]))):
            s = gpu_render(m, to_dev(cube), cam, mode, lut, **kw, **sm)
            for k in raw:
                assert np.array_equal(raw[k], s[k]), (mode, sm, k)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("mode", ["mip", "composite", "ratio"])
def test_smoothing_bricks(m, storage, mode):
    """Smoothing on the 16-bit bricks: the FP32 arithmetic on the rounded values."""
    dims = (70, 45, 66)
    cube = scene.tiny_cube(config_id=33, dims=dims, n_sources=3)
    c2 = scene.ratio_cube(cube, config_id=33)
    cam = scene.orbit_camera(dims, -25, 30, 80, 64)
    lut = scene.ratio_lut() if mode == "ratio" else scene.linear_lut()
    kw = _kw(mode)
    rnd = oracle.round_bf16 if storage == "bf16" else oracle.round_f16
    for sm in (_smooth("box2"), _smooth("taps9")):
        g = gpu_render(m, m.pack_bricks(to_dev(cube), storage), cam, mode, to_dev(lut),
                       vol2=m.pack_bricks(to_dev(c2), storage), **kw, **sm)
        o = oracle.render(rnd(cube), cam, mode, lut=lut, cube2=rnd(c2), eps_pos=1e-6, eps_val=1e-4, **kw, **sm)
        compare(g, o, mode, scale=_scale(cube, mode, o), tol=TOL_F32, max_fragile=0.05,
                what=f"{storage}/{mode}/{sm['smooth']}")


def test_smoothing_rejected_where_unsupported(m, ragged):
    import torch
    cube, _ = ragged
    cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 64, 48)
    lut = to_dev(scene.linear_lut())
    with pytest.raises(m.ShwError) as e:
        m.render(to_dev(cube), cam, "mip", lut=lut, smooth="box", smooth_arm=17)
    assert e.value.status == 1
    torch.cuda.synchronize()


@pytest.mark.parametrize("step", [0.5, 1.0])
@pytest.mark.parametrize("mode", ["mip", "avg", "composite", "moment1"])
def test_box_lattice_matches_direct(m, ragged, step, mode):
    """With a step of 1/2 voxel the box runs as running sums over the ray's own samples; it
    agrees with the direct per-sample sums (SHW_DEBUG_BOX_DIRECT) to FP32 rounding.  (A step of 1
    takes the direct sums either way.)"""
    cube, c2 = ragged
    cube = cube.copy()
    cube.reshape(-1)[np.random.default_rng(4).integers(0, cube.size, 40)] = np.nan  # windows with NaN taps
    cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 100, 75)
    lut = to_dev(scene.linear_lut())
    kw = dict(_kw(mode), step=step, smooth="box", smooth_arm=4)
    lat = gpu_render(m, to_dev(cube), cam, mode, lut, **kw)
    with m.debug_flags("box_direct"):
        dct = gpu_render(m, to_dev(cube), cam, mode, lut, **kw)
    scale = 1.0 if mode == "composite" else (float(cube.shape[0]) if mode == "moment1" else
                                              float(np.nanmax(cube) - np.nanmin(cube)))
    if mode != "composite":  # (compositing's exit sample is a rounding decision: oracle check only)
        assert np.array_equal(lat["nsamples"], dct["nsamples"])
        assert np.abs(lat["rgba"] - dct["rgba"]).max() <= TOL_F32
        assert np.nanmax(np.abs(lat["scalar"] - dct["scalar"])) <= TOL_F32 * scale
    o = oracle.render(cube, cam, mode, lut=scene.linear_lut(), eps_pos=1e-6, eps_val=1e-4, **kw)
    compare(lat, o, mode, scale=scale, max_fragile=0.05, what=f"lattice/{mode}/{step}")


def test_smoothing_edge_cases(m):
    """Degenerate inputs with in-ray smoothing: a single voxel (every tap clamps onto it), a
    one-channel slab, the eye inside the cube, a step longer than the cube (N = 0), and the
    line ratio of a single voxel on the pair storage."""
    lut = scene.linear_lut()
    kws = [dict(smooth="box", smooth_arm=3), dict(smooth="taps", smooth_taps=_taps("taps9"))]
    one = np.array([[[2.5]]], np.float32)
    cam = scene.orbit_camera((1, 1, 1), 10, 10, 17, 13)
    for sm in kws:
        g = gpu_render(m, to_dev(one), cam, "mip", to_dev(lut), **sm)
        o = oracle.render(one, cam, "mip", lut=lut, eps_pos=1e-6, **sm)
        compare(g, o, "mip", scale=1.0, what=f"1 voxel/{sm['smooth']}")
    slab = scene.tiny_cube(dims=(40, 30, 1), n_sources=1)
    cam = scene.orbit_camera((40, 30, 1), 20, 10, 24, 18)
    for sm in kws:
        g = gpu_render(m, to_dev(slab), cam, "avg", to_dev(lut), **sm)
        o = oracle.render(slab, cam, "avg", lut=lut, eps_pos=1e-6, **sm)
        compare(g, o, "avg", scale=float(slab.max() - slab.min()), max_fragile=1.0, what=f"slab/{sm['smooth']}")
    cube = scene.tiny_cube(dims=(48, 48, 48), n_sources=2)
    c = scene.orbit_camera((48, 48, 48), 20, 10, 64, 48, dist_scale=0.1)
    for sm in kws:
        for mode in ("mip", "composite"):
            g = gpu_render(m, to_dev(cube), c, mode, to_dev(lut), opacity_scale=0.05, **sm)
            o = oracle.render(cube, c, mode, lut=lut, opacity_scale=0.05, eps_pos=1e-6, eps_val=1e-4, **sm)
            compare(g, o, mode, scale=1.0 if mode == "composite" else float(cube.max() - cube.min()),
                    max_fragile=0.05, what=f"eye inside/{mode}/{sm['smooth']}")
        g = gpu_render(m, to_dev(cube), c, "mip", to_dev(lut), step=100.0, **sm)
        o = oracle.render(cube, c, "mip", lut=lut, step=100.0, eps_pos=1e-6, **sm)
        compare(g, o, "mip", scale=float(cube.max() - cube.min()), max_fragile=1.0, what=f"long step/{sm['smooth']}")
    pr = to_dev(np.stack([np.full((1, 1, 1), 2.0, np.float32), np.full((1, 1, 1), 1.0, np.float32)], axis=-1))
    g = gpu_render(m, pr, scene.orbit_camera((1, 1, 1), 10, 10, 9, 7), "ratio", to_dev(scene.ratio_lut()),
                   lo=0.0, hi=1.0, ratio_floor=0.5)
    hit = g["nsamples"] > 0
    assert hit.any() and np.all(g["scalar"][hit] == np.float32(0.5))
