"""GPU parity of shw_render (FP32 linear cube) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import scene
from parity import TOL_F32, compare, gpu_render, shw, to_dev

pytestmark = pytest.mark.gpu

MODES = ["mip", "avg", "composite", "spectral", "ratio", "moment1", "composite_spectral", "mip_rgb",
         "composite_rgb", "ratio_mip"]


@pytest.fixture(scope="module")
def m():
    return shw()


@pytest.fixture(scope="module")
def tiny():
    c = scene.tiny_cube()
    return c, scene.ratio_cube(c, config_id=1)


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
        return float(cube.shape[0])  # the moment is a height: its range is the channels
    return float(np.nanmax(cube) - np.nanmin(cube))


def test_ortho_nearest_mip_and_index_bit_exact(m, tiny):
    """Axis-aligned parallel view, nearest sampling: MIP = max over channels (Eq. 1), and the
    channel is the last maximum (Algorithm 4), bit-exact on GPU and oracle."""
    cube, _ = tiny
    cq = np.round(cube * 2).astype(np.float32)  # exact ties exercise the ">=" rule
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    lut = scene.linear_lut()
    g = gpu_render(m, to_dev(cq), cam, "spectral", to_dev(lut), interp="nearest")
    ref = cq.max(axis=0)[::-1].repeat(2, 0).repeat(2, 1)
    assert np.array_equal(g["scalar"], ref)
    last = (63 - np.argmax(cq[::-1], axis=0))[::-1].repeat(2, 0).repeat(2, 1)
    assert np.array_equal(g["index"], last)
    o = oracle.render(cq, cam, "spectral", interp="nearest", lut=lut)
    assert np.array_equal(g["scalar"].astype(np.float64), o["scalar"])
    assert np.array_equal(g["index"], o["index"])
    assert np.abs(g["rgba"] - o["rgba"]).max() <= TOL_F32


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_ortho_axis_parity(m, tiny, mode, interp):
    cube, c2 = tiny
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    lut = scene.ratio_lut() if mode.startswith("ratio") else scene.linear_lut()
    kw = _kw(mode)
    g = gpu_render(m, to_dev(cube), cam, mode, to_dev(lut), interp=interp, vol2=to_dev(c2), **kw)
    o = oracle.render(cube, cam, mode, interp=interp, lut=lut, cube2=c2, eps_pos=1e-6, eps_val=1e-4, **kw)
    exact = (mode in ("mip", "spectral", "ratio") and interp == "nearest")
    compare(g, o, mode, scale=_scale(cube, mode, o), exact=exact and mode != "ratio", what=f"{mode}/{interp}")


# ragged sizes: neither cube nor image a multiple of the 16x16 tile or of 32
RAGGED_DIMS = (61, 53, 47)


@pytest.fixture(scope="module")
def ragged():
    c = scene.tiny_cube(config_id=11, dims=RAGGED_DIMS, n_sources=4)
    return c, scene.ratio_cube(c, config_id=11)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
@pytest.mark.parametrize("view", ["persp", "ortho_oblique", "persp_steep"])
def test_general_view_parity(m, ragged, mode, interp, view):
    cube, c2 = ragged
    if view == "persp":
        cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 100, 75)
    elif view == "persp_steep":
        cam = scene.orbit_camera(RAGGED_DIMS, 137, -71, 83, 97, fov_deg=60)
    else:
        cam = scene.orbit_camera(RAGGED_DIMS, -52, 33, 90, 70, ortho=True)
    lut = scene.ratio_lut() if mode.startswith("ratio") else scene.linear_lut()
    kw = _kw(mode)
    g = gpu_render(m, to_dev(cube), cam, mode, to_dev(lut), interp=interp, vol2=to_dev(c2), **kw)
    o = oracle.render(cube, cam, mode, interp=interp, lut=lut, cube2=c2, eps_pos=1e-6, eps_val=1e-4, **kw)
    st = compare(g, o, mode, scale=_scale(cube, mode, o), what=f"{mode}/{interp}/{view}")
    assert (o["nsamples"] > 0).mean() > 0.2  # the view actually hits the cube


def test_composite_constant_cube_closed_form_gpu(m):
    lut = scene.linear_lut()
    v = -3.0 + 11.0 * 100 / 255
    cube = np.full((16, 12, 10), v, np.float32)
    cam = scene.ortho_axis_camera((10, 12, 16), 20, 24)
    s = 0.05
    g = gpu_render(m, to_dev(cube), cam, "composite", to_dev(lut), opacity_scale=s)
    vhat = (np.float64(np.float32(v)) + 3.0) / 11.0
    u = 255 * vhat
    i0 = int(np.floor(u)); f = u - i0
    col = (1 - f) * lut[i0].astype(np.float64) + f * lut[i0 + 1].astype(np.float64)
    A = 1 - (1 - s * col[3]) ** 32
    assert np.abs(g["rgba"][..., 3] - A).max() <= TOL_F32
    assert np.abs(g["rgba"][..., :3] - col[:3] * A).max() <= TOL_F32
    # early exit: opaque cube stops after the first sample pushing alpha over 0.99
    cube = np.full((64, 4, 4), 8.0, np.float32)
    cam = scene.ortho_axis_camera((4, 4, 64), 8, 8)
    g = gpu_render(m, to_dev(cube), cam, "composite", to_dev(lut), opacity_scale=0.3)
    k = next(k for k in range(1, 200) if 1 - 0.7 ** k > 0.99)
    assert (g["nsamples"] == k).all()


def test_edge_cases(m):
    lut = to_dev(scene.linear_lut())
    # a single voxel
    one = np.array([[[2.5]]], np.float32)
    cam = scene.orbit_camera((1, 1, 1), 10, 10, 17, 13)
    g = gpu_render(m, to_dev(one), cam, "mip", lut, interp="trilinear")
    o = oracle.render(one, cam, "mip", lut=scene.linear_lut(), eps_pos=1e-6)
    compare(g, o, "mip", scale=1.0, what="1 voxel")
    # a thin slab (1 channel) and a 1x1 image
    slab = scene.tiny_cube(dims=(40, 30, 1), n_sources=1)
    cam = scene.orbit_camera((40, 30, 1), 20, 10, 1, 1)
    g = gpu_render(m, to_dev(slab), cam, "avg", lut)
    o = oracle.render(slab, cam, "avg", lut=scene.linear_lut(), eps_pos=1e-6)
    compare(g, o, "avg", scale=float(slab.max() - slab.min()), max_fragile=1.0, what="1 channel")
    # the camera looking away: every ray misses
    c = scene.orbit_camera((32, 32, 32), 0, 0, 40, 30)
    c.fwd = -c.fwd
    c.right = -c.right
    g = gpu_render(m, to_dev(np.ones((32, 32, 32), np.float32)), c, "composite", lut)
    assert (g["rgba"] == 0).all() and (g["nsamples"] == 0).all() and (g["index"] == -1).all()
    # the eye inside the cube
    cube = scene.tiny_cube(dims=(48, 48, 48), n_sources=2)
    c = scene.orbit_camera((48, 48, 48), 20, 10, 64, 48, dist_scale=0.1)
    for mode in ("mip", "composite", "avg"):
        g = gpu_render(m, to_dev(cube), c, mode, lut, opacity_scale=0.05)
        o = oracle.render(cube, c, mode, lut=scene.linear_lut(), opacity_scale=0.05, eps_pos=1e-6, eps_val=1e-4)
        compare(g, o, mode, scale=1.0 if mode == "composite" else float(cube.max() - cube.min()),
                what=f"eye inside/{mode}")
    # a step longer than the cube: N = 0 for most rays
    g = gpu_render(m, to_dev(cube), c, "mip", lut, step=100.0)
    o = oracle.render(cube, c, "mip", lut=scene.linear_lut(), step=100.0, eps_pos=1e-6)
    compare(g, o, "mip", scale=float(cube.max() - cube.min()), max_fragile=1.0, what="long step")


def test_nan_voxels_are_datamin(m, tiny):
    cube = tiny[0].copy()
    cube[:, 10, 10] = np.nan
    cube[5:9, 20:30, 20] = np.nan
    cam = scene.orbit_camera((64, 64, 64), 25, 15, 96, 80)
    lut = scene.linear_lut()
    for mode in ("mip", "avg", "composite"):
        g = gpu_render(m, to_dev(cube), cam, mode, to_dev(lut), opacity_scale=0.05)
        o = oracle.render(cube, cam, mode, lut=lut, opacity_scale=0.05, eps_pos=1e-6, eps_val=1e-4)
        assert np.isfinite(g["rgba"]).all() and np.isfinite(g["scalar"]).all()
        compare(g, o, mode, scale=1.0 if mode == "composite" else float(np.nanmax(cube) - np.nanmin(cube)),
                what=f"nan/{mode}")


def test_deterministic(m, ragged):
    cube, c2 = ragged
    cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 100, 75)
    lut = to_dev(scene.linear_lut())
    ct = to_dev(cube)
    for mode in MODES:
        kw = _kw(mode)
        a = gpu_render(m, ct, cam, mode, lut, vol2=to_dev(c2), **kw)
        b = gpu_render(m, ct, cam, mode, lut, vol2=to_dev(c2), **kw)
        for k in a:
            assert np.array_equal(a[k], b[k]), (mode, k)


def test_launch_counter_moves(m, tiny):
    before = m.launch_count()
    gpu_render(m, to_dev(tiny[0]), scene.ortho_axis_camera((64, 64, 64), 128, 128), "mip",
               to_dev(scene.linear_lut()))
    assert m.launch_count() == before + 1


FILTER_CASES = [("clip", -0.5, 3.0), ("scale", -1.0, 4.0)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("filt", range(len(FILTER_CASES)))
@pytest.mark.parametrize("view", ["axis", "persp"])
def test_filters_parity(m, ragged, tiny, mode, filt, view):
    """Per-sample intensity clipping (Algorithm 10) and domain scaling (Algorithm 11)."""
    kind, tmin, tmax = FILTER_CASES[filt]
    if view == "axis":
        cube, c2 = tiny
        cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    else:
        cube, c2 = ragged
        cam = scene.orbit_camera(RAGGED_DIMS, 30, 20, 100, 75)
    lut = scene.ratio_lut() if mode.startswith("ratio") else scene.linear_lut()
    kw = _kw(mode)
    if kind == "scale" and not mode.startswith("ratio"):
        kw.update(lo=-0.5, hi=1.0)  # the scaled domain is [0, 1]; DATAMIN below it
    if mode.startswith("ratio"):
        tmin, tmax = 0.5, 6.0
    f = dict(filter=kind, min_threshold=tmin, max_threshold=tmax)
    g = gpu_render(m, to_dev(cube), cam, mode, to_dev(lut), vol2=to_dev(c2), **kw, **f)
    o = oracle.render(cube, cam, mode, lut=lut, cube2=c2, eps_pos=1e-6, eps_val=1e-4, **kw, **f)
    compare(g, o, mode, scale=_scale(cube, mode, o), max_fragile=0.05, what=f"{mode}/{kind}/{view}")


@pytest.mark.parametrize("mode", ["spectral", "moment1"])
def test_alpha_threshold_parity(m, ragged, mode):
    cube, _ = ragged
    cam = scene.orbit_camera(RAGGED_DIMS, -40, 25, 90, 70)
    lut = scene.linear_lut()
    f = dict(alpha_threshold=True, min_threshold=2.0 if mode == "spectral" else 0.0)
    g = gpu_render(m, to_dev(cube), cam, mode, to_dev(lut), **f)
    o = oracle.render(cube, cam, mode, lut=lut, eps_pos=1e-6, eps_val=1e-4, **f)
    compare(g, o, mode, scale=_scale(cube, mode, o), max_fragile=0.05, what=f"{mode}/alpha-threshold")
    a = g["rgba"][..., 3]
    assert set(np.unique(a)) <= {0.0, 1.0} and (a == 1.0).any() and (a == 0.0).any()


def test_render_refuses_a_capturing_stream(m):
    """A render's persistent CTAs take tiles from a work counter handed out at call time, so a
    call made while the stream is captured into a CUDA graph is refused (SHW_EUNSUPPORTED)
    before anything is enqueued; batch plans are the graph-launched form."""
    cube = to_dev(scene.tiny_cube())
    lut = to_dev(scene.linear_lut())
    cam = scene.orbit_camera((64, 64, 64), 30, 20, 32, 24)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = []
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        try:
            m.render(cube, cam, "mip", lut=lut)
        except m.ShwError as e:
            status.append(e.status)
    assert status == [2]
    m.sync_status()
