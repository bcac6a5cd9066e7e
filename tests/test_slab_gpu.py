"""The staged marcher (slabs of the cube staged in shared memory by tensor copies) on the GPU.

It runs the gather marcher's arithmetic on the same fixed-point sample positions, so every
output -- image, scalar, channel, sample count, compositing checkpoints -- must equal the
gather marcher's bit for bit, for views whose major axis is x, y or z, in both directions,
parallel and perspective, with the eye outside or inside the cube; and match the FP64 oracle.
The linear 16-bit storages hold the same rounded values as the 16-bit bricks, so their
renders must equal the brick renders bit for bit.  SHW_DEBUG_REQUIRE_STAGING makes a request
the staged marcher does not serve fail instead of falling back, so each comparison is known
to have used it."""
import numpy as np
import pytest
import torch

import oracle
import scene
from parity import TOL_F32, compare, gpu_render, shw, to_dev

pytestmark = pytest.mark.gpu

SINGLE = ["mip", "avg", "composite", "spectral", "moment1", "composite_spectral", "mip_rgb", "composite_rgb"]
VIEWS = [
    dict(dims=(68, 45, 66), yaw=30, pitch=20, W=100, H=75),               # z-major, oblique
    dict(dims=(68, 45, 66), yaw=80, pitch=10, W=90, H=61),                # x-major
    dict(dims=(68, 45, 66), yaw=15, pitch=75, W=70, H=83),                # y-major, looking down
    dict(dims=(68, 45, 66), yaw=200, pitch=-35, W=77, H=77),              # negative directions
    dict(dims=(64, 40, 96), yaw=30, pitch=20, W=160, H=90, ortho=True),   # parallel, oblique
    dict(dims=(64, 40, 96), yaw=-135, pitch=40, W=49, H=33, dist_scale=0.3),  # eye inside the cube
]


@pytest.fixture(scope="module")
def m():
    return shw()


def _cam(v):
    return scene.orbit_camera(v["dims"], v["yaw"], v["pitch"], v["W"], v["H"], ortho=v.get("ortho", False),
                              dist_scale=v.get("dist_scale", 1.0))


def _cube(i, dims):
    cube = scene.tiny_cube(config_id=90 + i, dims=dims, n_sources=3)
    cube[dims[2] // 3, dims[1] // 2, dims[0] // 4] = np.nan
    return cube


def _kw(mode):
    return dict(opacity_scale=0.05) if mode.startswith("composite") else {}


def _render(m, vol, cam, mode, lut, flags=(), **kw):
    with m.debug_flags(*flags):
        out = m.render(vol, cam, mode, lut=lut, **kw)
        torch.cuda.synchronize()
    m.sync_status()
    return out


def _same(a, b, what):
    assert set(a) == set(b), what
    for k in a:
        assert torch.equal(a[k], b[k]), (k, what)


@pytest.mark.parametrize("view", range(len(VIEWS)))
@pytest.mark.parametrize("mode", SINGLE)
def test_staged_equals_gather(m, view, mode):
    v = VIEWS[view]
    cube_t = to_dev(_cube(view, v["dims"]))
    lut = to_dev(scene.linear_lut())
    cam = _cam(v)
    kw = _kw(mode)
    if mode == "composite":
        kw.update(ckpt=True, ckpt_interval=9)
    a = _render(m, cube_t, cam, mode, lut, ("require_staging",), **kw)
    b = _render(m, cube_t, cam, mode, lut, ("no_staging",), **kw)
    ca, cb = a.pop("ckpt", None), b.pop("ckpt", None)
    _same(a, b, f"view {view} {mode}")
    assert int(a["nsamples"].max()) > 0
    if ca is not None:
        H, W = cam.height, cam.width
        ka = ca[:4 * H * W].view(torch.int32).reshape(H, W)
        assert torch.equal(ka, cb[:4 * H * W].view(torch.int32).reshape(H, W))
        ta = ca[4 * H * W:].view(torch.float32).reshape(-1, H, W)
        tb = cb[4 * H * W:].view(torch.float32).reshape(-1, H, W)
        used = torch.arange(ta.shape[0], device="cuda")[:, None, None] < (ka[None] + 8) // 9
        assert torch.equal(ta[used], tb[used])


@pytest.mark.parametrize("view", [0, 1, 2, 4, 5])
@pytest.mark.parametrize("mode", ["mip", "avg", "composite", "spectral", "moment1"])
def test_staged_matches_oracle(m, view, mode):
    v = VIEWS[view]
    cube = _cube(view, v["dims"])
    cam = _cam(v)
    kw = _kw(mode)
    with m.debug_flags("require_staging"):
        g = gpu_render(m, to_dev(cube), cam, mode, to_dev(scene.linear_lut()), **kw)
    o = oracle.render(cube, cam, mode, lut=scene.linear_lut(), eps_pos=1e-6, eps_val=1e-4, **kw)
    scale = float(v["dims"][2]) if mode == "moment1" else (
        1.0 if mode == "composite" else float(np.nanmax(cube) - np.nanmin(cube)))
    compare(g, o, mode, scale=scale, max_fragile=0.05, what=f"staged/{view}/{mode}")


def test_staged_early_exit(m):
    """Compositing stops the ray after the sample that makes alpha > 0.99, inside a slab."""
    dims = (48, 40, 56)
    cube = np.full(dims[::-1], 8.0, np.float32)
    cam = scene.orbit_camera(dims, 25, 15, 64, 48)
    lut = to_dev(scene.linear_lut())
    a = _render(m, to_dev(cube), cam, "composite", lut, ("require_staging",), opacity_scale=0.3)
    b = _render(m, to_dev(cube), cam, "composite", lut, ("no_staging",), opacity_scale=0.3)
    _same(a, b, "early exit")
    k = next(k for k in range(1, 200) if 1 - 0.7 ** k > 0.99)
    ns = a["nsamples"].cpu().numpy()
    assert ns.max() == k


@pytest.mark.parametrize("mode", ["ratio", "ratio_mip"])
def test_staged_pair_storage(m, mode):
    """The line ratios on the float32 pair storage: staged equals the gather marcher."""
    dims = (68, 45, 66)
    cube = scene.tiny_cube(config_id=97, dims=dims, n_sources=3)
    c2 = scene.ratio_cube(cube, config_id=97)
    pair = torch.stack([to_dev(cube), to_dev(c2)], dim=-1).contiguous()
    lut = to_dev(scene.ratio_lut())
    kw = dict(lo=0.0, hi=1.0, ratio_floor=1.0)
    for v in (VIEWS[0], VIEWS[1], VIEWS[4]):
        cam = _cam(v) if v["dims"] == dims else scene.orbit_camera(dims, v["yaw"], v["pitch"], v["W"], v["H"],
                                                                   ortho=v.get("ortho", False))
        a = _render(m, pair, cam, mode, lut, ("require_staging",), **kw)
        b = _render(m, pair, cam, mode, lut, ("no_staging",), **kw)
        _same(a, b, f"pair {mode}")
        c = _render(m, to_dev(cube), cam, mode, lut, (), vol2=to_dev(c2), **kw)
        _same(a, c, f"pair vs two cubes {mode}")


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("mode", SINGLE)
def test_linear16_equals_bricks(m, storage, mode):
    """A linear 16-bit cube holds the bricks' rounded values: identical renders (x rows of 72
    values: 16-byte multiples)."""
    v = dict(VIEWS[0], dims=(72, 45, 66))
    cube_t = to_dev(_cube(0, v["dims"]))
    lut = to_dev(scene.linear_lut())
    cam = _cam(v)
    lin = m.pack_bricks(cube_t, storage + "_linear")
    assert lin.data.numel() == cube_t.numel()
    a = _render(m, lin, cam, mode, lut, (), **_kw(mode))
    b = _render(m, m.pack_bricks(cube_t, storage), cam, mode, lut, (), **_kw(mode))
    _same(a, b, f"{storage} linear vs bricks {mode}")


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("mode", ["ratio", "ratio_mip"])
def test_linear16_pairs_equal_pair_bricks(m, storage, mode):
    dims = (68, 45, 66)
    cube = scene.tiny_cube(config_id=98, dims=dims, n_sources=3)
    c2 = scene.ratio_cube(cube, config_id=98)
    pair = torch.stack([to_dev(cube), to_dev(c2)], dim=-1).contiguous()
    lut = to_dev(scene.ratio_lut())
    kw = dict(lo=0.0, hi=1.0, ratio_floor=1.0)
    cam = _cam(VIEWS[1])
    a = _render(m, m.pack_bricks(pair, storage + "_linear"), cam, mode, lut, (), **kw)
    b = _render(m, m.pack_bricks(pair, storage), cam, mode, lut, (), **kw)
    _same(a, b, f"{storage} linear pairs vs pair bricks {mode}")


def test_linear16_conversion_rounds_to_nearest_even(m):
    cube = scene.tiny_cube(config_id=99, dims=(40, 8, 8), n_sources=1)
    ct = to_dev(cube)
    for storage, rnd in (("bf16", oracle.round_bf16), ("f16", oracle.round_f16)):
        lin = m.pack_bricks(ct, storage + "_linear")
        torch.cuda.synchronize()
        raw = lin.data.cpu().numpy().view(np.uint16).astype(np.uint32)
        if storage == "bf16":
            vals = (raw << 16).view(np.float32)
        else:
            vals = raw.astype(np.uint16).view(np.float16).astype(np.float32)
        assert np.array_equal(vals.reshape(cube.shape), rnd(cube).astype(np.float32))


def test_staged_refusals_and_fallbacks(m):
    """Requests the staged marcher does not serve: with SHW_DEBUG_REQUIRE_STAGING they are
    refused; without it a float32 cube takes the gather marcher, a linear 16-bit cube is
    refused (no other marcher reads it)."""
    lut = to_dev(scene.linear_lut())
    dims = (66, 40, 50)  # 66 x 4 bytes is not a 16-byte multiple
    cube_t = to_dev(scene.tiny_cube(config_id=91, dims=dims, n_sources=2))
    cam = scene.orbit_camera(dims, 30, 20, 40, 30)
    with m.debug_flags("require_staging"), pytest.raises(m.ShwError) as e:
        m.render(cube_t, cam, "mip", lut=lut)
    assert e.value.status == 2
    a = _render(m, cube_t, cam, "mip", lut, ())
    b = _render(m, cube_t, cam, "mip", lut, ("no_staging",))
    _same(a, b, "ragged nx")
    lin = m.pack_bricks(to_dev(scene.tiny_cube(config_id=91, dims=(64, 40, 50), n_sources=2)), "bf16_linear")
    cam2 = scene.orbit_camera((64, 40, 50), 30, 20, 40, 30)
    for kw in (dict(interp="nearest"), dict(smooth="box", smooth_arm=1)):
        with pytest.raises(m.ShwError) as e:
            m.render(lin, cam2, "mip", lut=lut, **kw)
        assert e.value.status == 2
    with pytest.raises(m.ShwError) as e:  # nearest sampling is the gather marcher's
        with m.debug_flags("require_staging"):
            m.render(to_dev(scene.tiny_cube(config_id=91, dims=(64, 40, 50), n_sources=2)), cam2, "mip", lut=lut,
                     interp="nearest")
    assert e.value.status == 2
    torch.cuda.synchronize()


@pytest.mark.parametrize("view", [0, 1, 2, 4])
def test_staged_mip_without_channel(m, view):
    """MIP with no channel output keeps the running maximum alone (the staged marcher's
    value-only instance); image and maximum equal the gather marcher's."""
    v = VIEWS[view]
    cube_t = to_dev(_cube(view, v["dims"]))
    lut = to_dev(scene.linear_lut())
    cam = _cam(v)
    a = _render(m, cube_t, cam, "mip", lut, ("require_staging",), index=False)
    b = _render(m, cube_t, cam, "mip", lut, ("no_staging",), index=False)
    assert "index" not in a
    _same(a, b, f"mip value-only view {view}")
